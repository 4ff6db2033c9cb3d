"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source: a dropped term, a wrong
sign, constant, count or index, or a transposed operand.  The copy is compiled into a
temporary directory and loaded in place of the oracle.  The pin meant to catch that
mistake must then fail; the same pin passes on the real oracle in the other
``test_oracle_*`` files.  The oracle's own source is never modified, and every planted
mistake keeps each memory access in bounds.
"""
import concurrent.futures as cf
import contextlib
import os
import subprocess

import pytest

import oracle
import test_oracle_conditionals as cond
import test_oracle_hyper as hyper
import test_oracle_rng as rng
import test_oracle_sampler as sampler


def _kat_all():
    for ctr, key, expect in rng._kat():
        rng.test_philox_known_answers(ctr, key, expect)


# (name, text in the oracle source, planted replacement, pin that must fail)
MUTANTS = [
    ("philox: nine rounds", "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {",
     _kat_all),
    ("philox: key schedule constant", "k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;", _kat_all),
    ("philox: multipliers exchanged", "(uint64_t)0xD2511F53u * (uint64_t)x0",
     "(uint64_t)0xCD9E8D57u * (uint64_t)x0", _kat_all),
    ("box-muller: cos and sin exchanged", "*zc = rho * cos(th);\n    *zs = rho * sin(th);",
     "*zc = rho * sin(th);\n    *zs = rho * cos(th);", rng.test_normal_stream_box_muller_identity),
    ("box-muller: radius without the factor 2", "sqrt(-2.0 * log(u_open(wa)))",
     "sqrt(-log(u_open(wa)))", rng.test_normal_stream_box_muller_identity),
    ("gamma: d = a - 1/2", "double d = a - 1.0 / 3.0;", "double d = a - 0.5;",
     lambda: rng.test_gamma_moments(1.0)),
    ("gamma: acceptance test with d v and d exchanged",
     "log(u) < 0.5 * x * x + d - d * v + d * log(v)",
     "log(u) < 0.5 * x * x - d + d * v + d * log(v)", rng.test_gamma_ks_and_acceptance),
    ("cholesky: transposed index in the update", "s -= L[i * K + k] * L[j * K + k];",
     "s -= L[k * K + i] * L[j * K + k];", lambda: cond.test_cholesky_matches_lapack(5)),
    ("back solve: L instead of its transpose",
     "for (int k = i + 1; k < K; ++k) s -= L[k * K + i] * x[k];",
     "for (int k = i + 1; k < K; ++k) s -= L[i * K + k] * x[k];",
     lambda: cond.test_spd_inverse_matches_numpy(3)),
    ("row statistics: scatter over n - 1", "for (int i = 0; i < K * K; ++i) S[i] /= (double)n;",
     "for (int i = 0; i < K * K; ++i) S[i] /= (double)(n - 1);", cond.test_row_stats_match_numpy),
    ("conditional: prior mean term dropped", "for (int k = 0; k < K; ++k) b[k] = LamMu[k];",
     "for (int k = 0; k < K; ++k) b[k] = 0.0;", lambda: cond.test_row_conditional_closed_form(3, 0)),
    ("conditional: alpha dropped from the Gram", "Lam[a * K + c] += alpha * yc[a] * yc[c];",
     "Lam[a * K + c] += yc[a] * yc[c];", lambda: cond.test_row_conditional_closed_form(3, 2)),
    ("conditional: alpha dropped from the right-hand side", "b[a] += alpha * val[t] * yc[a];",
     "b[a] += val[t] * yc[a];", lambda: cond.test_row_conditional_closed_form(3, 2)),
    ("conditional: noise through L^-1 instead of L^-T", "solve_upper_t(K, L, z, e);",
     "solve_lower(K, L, z, e);", lambda: cond.test_row_conditional_closed_form(3, 2)),
    ("conditional: a rating paired with the previous rating's factor row",
     "const double* yc = Y + (size_t)idx[t] * K;",
     "const double* yc = Y + (size_t)idx[t > 0 ? t - 1 : 0] * K;",
     lambda: cond.test_row_conditional_closed_form(3, 2)),
    ("normal-wishart: nu* without n", "double beta_s = beta0 + nd, nu_s = nu0 + nd;",
     "double beta_s = beta0 + nd, nu_s = nu0;", hyper.test_wishart_moments_and_mean_draw),
    ("normal-wishart: beta* without n", "double beta_s = beta0 + nd, nu_s = nu0 + nd;",
     "double beta_s = beta0, nu_s = nu0 + nd;", hyper.test_wishart_moments_and_mean_draw),
    ("normal-wishart: scatter not scaled by n", "nd * S[a * K + b]", "S[a * K + b]",
     hyper.test_wishart_moments_and_mean_draw),
    ("normal-wishart: prior-mean cross term dropped",
     "cross * (mu0[a] - xbar[a]) * (mu0[b] - xbar[b])",
     "0.0 * (mu0[a] - xbar[a]) * (mu0[b] - xbar[b])", hyper.test_wishart_moments_and_mean_draw),
    ("normal-wishart: Bartlett diagonal degrees of freedom off by one",
     "0.5 * (nu_s - (double)k)", "0.5 * (nu_s - (double)k - 1.0)",
     hyper.test_wishart_moments_and_mean_draw),
    ("normal-wishart: B = A L_W (operands transposed)", "s += LW[i * K + k] * A[k * K + j];",
     "s += A[i * K + k] * LW[k * K + j];", hyper.test_wishart_moments_and_mean_draw),
    ("normal-wishart: mean precision without beta*", "tmp[i] = beta_s * Lambda[i];",
     "tmp[i] = Lambda[i];", hyper.test_wishart_moments_and_mean_draw),
    ("centring: mean over nnz - 1 ratings", "total / (double)nnz", "total / (double)(nnz - 1)",
     sampler.test_centering_uses_training_mean),
    ("predict: training mean not added back", "double p = o->rbar;", "double p = 0.0;",
     sampler.test_predict_matches_brute_force),
    ("predict: running average starts one sweep late", ">= (int64_t)o->burn_in",
     "> (int64_t)o->burn_in", sampler.test_predict_matches_brute_force),
    ("column view: ratings attributed to the mirrored user", "mv->idx[p] = (int32_t)i;",
     "mv->idx[p] = (int32_t)(M - 1 - i);", sampler.test_planted_converges_to_noise_floor),
]


def _compile(src_text, old, new, out_dir, n):
    assert src_text.count(old) == 1, old
    path = os.path.join(out_dir, "mutant%02d.c" % n)
    with open(path, "w") as f:
        f.write(src_text.replace(old, new))
    lib = os.path.join(out_dir, "libmutant%02d.so" % n)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", path, "-o", lib, "-lm"],
                   check=True)
    return lib


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(oracle._SRC).read()
    out = str(tmp_path_factory.mktemp("oracle_mutants"))
    with cf.ThreadPoolExecutor(8) as ex:
        libs = list(ex.map(lambda a: _compile(src, a[1][1], a[1][2], out, a[0]), enumerate(MUTANTS)))
    return {m[0]: lib for m, lib in zip(MUTANTS, libs)}


@contextlib.contextmanager
def _loaded(path):
    """The oracle module's routines run on the library at `path` inside the block."""
    saved_lib, saved_build = oracle._lib, oracle.build
    oracle._lib = None
    oracle.build = lambda force=False: path
    try:
        oracle.lib()
        yield
    finally:
        oracle.build = saved_build
        oracle._lib = saved_lib


@pytest.mark.parametrize("name,pin", [(m[0], m[3]) for m in MUTANTS], ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(mutant_libs, name, pin):
    with _loaded(mutant_libs[name]):
        with pytest.raises((AssertionError, RuntimeError, ArithmeticError, ValueError)):
            pin()


def test_unchanged_source_passes_the_same_pins(tmp_path):
    # the harness itself: the oracle compiled the same way, untouched, passes a sample of
    # the pins above (so a failure there comes from the planted mistake)
    src = open(oracle._SRC).read()
    lib = _compile(src, "for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 10; ++r) {",
                   str(tmp_path), 99)
    with _loaded(lib):
        _kat_all()
        cond.test_row_conditional_closed_form(3, 2)
        sampler.test_predict_matches_brute_force()
