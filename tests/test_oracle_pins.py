"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a
hand-worked example, brute-force loops on tiny inputs, closed forms,
invariants, least-squares optimality, or a special case that reduces to a
textbook algorithm.  A plausible slip in the oracle (a dropped term, a wrong
index or sign, a transposed operand) fails at least one of them.
"""

import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import ppl_oracle as orc
from paper_2503_10380_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _brute_R(Bvv, tau):
    X, v, _ = Bvv.shape
    o = tau.shape[0]
    R = np.zeros((v, v, o, o))
    for a, b, i, j in itertools.product(range(v), range(v), range(o), range(o)):
        s = 0.0
        for Q, c, d in itertools.product(range(X), range(v), range(v)):
            s += Bvv[Q, a, c] * Bvv[Q, b, d] * tau[i, j, c, d]
        R[a, b, i, j] = s
    return R


@pytest.fixture(scope="module")
def tiny():
    return inputs.make_inputs(o=3, v=5, X=4, R=6, seed=7)


# ---------------------------------------------------------------- golden

def test_hand_worked_example():
    d = json.load(open(os.path.join(GOLDEN, "hand_o2v2.json")))
    B = np.array(d["B"], dtype=np.float64)
    tau = np.array(d["tau"], dtype=np.float64)
    o = d["o"]
    Rt = orc.ppl_tensor(B[:, o:, o:], tau)
    assert np.array_equal(Rt, np.array(d["R_abij"], dtype=np.float64))
    n2, E = orc.exact_contract(B, tau, o)
    assert n2 == d["normR2"] and E == d["E_exact"]
    assert orc.energy_of_tensor(Rt, B, o) == d["E_exact"]
    U = {m: np.ones((2, 1)) for m in orc.MODES}
    for m in orc.MODES:
        assert np.array_equal(orc.mttkrp(B[:, o:, o:], tau, U, m)[:, 0], d["ones_mttkrp"])
    lam = np.ones(1)
    assert orc.cp_norm2(U, lam) == d["ones_cp_norm2"]
    assert orc.energy_cp(B, o, U, lam) == d["ones_cp_energy"]


# ---------------------------------------------------------------- the tensor

def test_ppl_tensor_matches_bruteforce_loops():
    inp = inputs.make_inputs(o=2, v=3, X=2, R=2, seed=3)
    assert _rel(orc.ppl_tensor(inp.Bvv, inp.tau), _brute_R(inp.Bvv, inp.tau)) < 1e-14


def test_pair_symmetry_of_R(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    assert _rel(Rt, Rt.transpose(1, 0, 3, 2)) < 1e-13
    # an input without pair symmetry breaks it: the invariant is not vacuous
    tau_bad = tiny.tau.copy()
    tau_bad[0, 1] += 0.5
    Rb = orc.ppl_tensor(tiny.Bvv, tau_bad)
    assert _rel(Rb, Rb.transpose(1, 0, 3, 2)) > 1e-3


def test_exact_rows_match_formed_tensor(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    rows, n2, E = orc.exact_rows(tiny.B, tiny.tau, tiny.o, range(tiny.v))
    assert _rel(rows, Rt.transpose(0, 1, 2, 3)) < 1e-13
    assert abs(n2 - float(np.sum(Rt * Rt))) < 1e-12 * n2
    assert abs(E - orc.energy_of_tensor(Rt, tiny.B, tiny.o)) < 1e-12 * abs(E)


def test_energy_of_tensor_bruteforce(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    o, v = tiny.o, tiny.v
    Bov = tiny.Bov
    E = 0.0
    for a, b, i, j in itertools.product(range(v), range(v), range(o), range(o)):
        giajb = float(np.dot(Bov[:, i, a], Bov[:, j, b]))
        gibja = float(np.dot(Bov[:, i, b], Bov[:, j, a]))
        E += Rt[a, b, i, j] * (2.0 * giajb - gibja)
    assert abs(E - orc.energy_of_tensor(Rt, tiny.B, o)) < 1e-13 * abs(E)


# ---------------------------------------------------------------- MTTKRP

def test_explicit_mttkrp_bruteforce(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    U = tiny.factors
    v, o, R = tiny.v, tiny.o, tiny.R
    M = np.zeros((o, R))
    for i, r in itertools.product(range(o), range(R)):
        M[i, r] = sum(Rt[a, b, i, j] * U["a"][a, r] * U["b"][b, r] * U["j"][j, r]
                      for a in range(v) for b in range(v) for j in range(o))
    assert _rel(orc.mttkrp_explicit(Rt, U, "i"), M) < 1e-13


@pytest.mark.parametrize("mode", orc.MODES)
def test_matrix_free_mttkrp_equals_explicit(tiny, mode):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    M_free = orc.mttkrp(tiny.Bvv, tiny.tau, tiny.factors, mode)
    M_expl = orc.mttkrp_explicit(Rt, tiny.factors, mode)
    assert _rel(M_free, M_expl) < 1e-12


def test_matrix_free_mttkrp_ragged_shapes():
    inp = inputs.make_inputs(o=1, v=7, X=3, R=1, seed=11)
    Rt = orc.ppl_tensor(inp.Bvv, inp.tau)
    for m in orc.MODES:
        assert _rel(orc.mttkrp(inp.Bvv, inp.tau, inp.factors, m),
                    orc.mttkrp_explicit(Rt, inp.factors, m)) < 1e-12


# ---------------------------------------------------------------- solve

def test_cholesky_clamped_spd_matches_library():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 30))
    V = A @ A.T + 30 * np.eye(30)
    L, nc = orc.cholesky_clamped(V)
    assert nc == 0
    assert _rel(L, np.linalg.cholesky(V)) < 1e-14


def test_cholesky_clamped_singular_counts_and_stays_finite():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((12, 4))
    V = A @ A.T                       # rank 4
    L, nc = orc.cholesky_clamped(V)
    assert nc == 8
    assert np.all(np.isfinite(L))
    # the factorisation reproduces V up to the clamped pivots
    assert np.max(np.abs(L @ L.T - V)) < 1e-10 * np.max(np.abs(V))


@pytest.mark.parametrize("mode", orc.MODES)
def test_update_is_least_squares_solution(tiny, mode):
    """The normal-equation update M V^{-1} equals the least-squares solution of
    the unfolded problem min ||R_(n) - U K^T||, K the Khatri-Rao product."""
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    U = tiny.factors
    axes = {"a": 0, "b": 1, "i": 2, "j": 3}
    n = axes[mode]
    others = [m for m in orc.MODES if m != mode]
    Rn = np.moveaxis(Rt, n, 0).reshape(Rt.shape[n], -1)
    K = np.einsum("xr,yr,zr->xyzr", *[U[m] for m in others]).reshape(-1, tiny.R)
    U_ls = np.linalg.lstsq(K, Rn.T, rcond=None)[0].T
    M = orc.mttkrp(tiny.Bvv, tiny.tau, U, mode)
    Ut, nc = orc.solve_normal(M, orc.hadamard_v(U, mode))
    assert nc == 0
    assert _rel(Ut, U_ls) < 1e-9


def test_each_mode_update_does_not_increase_residual(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    U = {m: tiny.factors[m].copy() for m in orc.MODES}
    lam = np.ones(tiny.R)
    prev = np.inf
    for _ in range(4):
        for mode in orc.MODES:
            M = orc.mttkrp(tiny.Bvv, tiny.tau, U, mode)
            Ut, _ = orc.solve_normal(M, orc.hadamard_v(U, mode))
            U[mode], lam = orc.normalise(Ut)
            res = float(np.linalg.norm(Rt - orc.reconstruct(U, lam)))
            assert res <= prev * (1 + 1e-10)
            prev = res


def test_planted_rank_is_recovered():
    """X = 1 and tau = sum_s p_s x q_s x u_s x w_s give R of CP rank <= S X;
    ALS at rank S X reaches fit > 1 - 1e-10."""
    o, v, X, S = 3, 4, 1, 2
    rng = np.random.default_rng(5)
    Bvv = rng.standard_normal((X, v, v))
    Bvv = Bvv + Bvv.transpose(0, 2, 1)
    p, q = rng.standard_normal((S, o)), rng.standard_normal((S, o))
    u, w = rng.standard_normal((S, v)), rng.standard_normal((S, v))
    tau = np.einsum("si,sj,sc,sd->ijcd", p, q, u, w)
    Rt = orc.ppl_tensor(Bvv, tau)
    normR2 = float(np.sum(Rt * Rt))
    U0 = {m: rng.standard_normal((o if m in "ij" else v, S * X)) for m in orc.MODES}
    U, lam, hist = orc.cp_als(Bvv, tau, U0, 300, normR2)
    # the explicit residual: the expansion ||R||^2 - 2<R,R~> + ||R~||^2 cancels
    # to rounding level (about 1e-8 after the square root) near fit = 1
    fit_explicit = 1 - np.linalg.norm(Rt - orc.reconstruct(U, lam)) / math.sqrt(normR2)
    assert fit_explicit > 1 - 1e-10
    assert hist[-1]["fit"] > 1 - 1e-7


def test_rank_one_als_is_higher_order_power_method(tiny):
    """At R = 1 each ALS update is u_n = R x_{m != n} u_m, normalised: the
    higher-order power method (De Lathauwer, De Moor, Vandewalle 2000)."""
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    U0 = {m: tiny.factors[m][:, :1].copy() for m in orc.MODES}
    U, lam, _ = orc.cp_als(tiny.Bvv, tiny.tau, U0, 3)
    h = {m: U0[m][:, 0].copy() for m in orc.MODES}
    for _ in range(3):
        h["a"] = np.tensordot(np.tensordot(np.tensordot(Rt, h["j"], ([3], [0])), h["i"], ([2], [0])), h["b"], ([1], [0]))
        s = np.linalg.norm(h["a"]); h["a"] /= s
        h["b"] = np.tensordot(np.tensordot(np.tensordot(Rt, h["j"], ([3], [0])), h["i"], ([2], [0])), h["a"], ([0], [0]))
        s = np.linalg.norm(h["b"]); h["b"] /= s
        h["i"] = np.tensordot(np.tensordot(np.tensordot(Rt, h["j"], ([3], [0])), h["b"], ([1], [0])), h["a"], ([0], [0]))
        s = np.linalg.norm(h["i"]); h["i"] /= s
        h["j"] = np.tensordot(np.tensordot(np.tensordot(Rt, h["i"], ([2], [0])), h["b"], ([1], [0])), h["a"], ([0], [0]))
        s = np.linalg.norm(h["j"]); h["j"] /= s
    for m in orc.MODES:
        assert _rel(U[m][:, 0], h[m]) < 1e-12
    assert abs(lam[0] - s) < 1e-12 * s


# ---------------------------------------------------------------- fit, eta, norms

def test_cp_norm2_closed_form(tiny):
    lam = np.linspace(0.5, 2.0, tiny.R)
    Rt = orc.reconstruct(tiny.factors, lam)
    assert abs(orc.cp_norm2(tiny.factors, lam) - float(np.sum(Rt * Rt))) < 1e-12 * float(np.sum(Rt * Rt))


def test_fit_and_eta_against_formed_tensors(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    normR2 = float(np.sum(Rt * Rt))
    U0 = tiny.factors
    lam0 = np.ones(tiny.R)
    U1, lam1, info = orc.als_sweep(tiny.Bvv, tiny.tau, U0, lam0, normR2)
    R1 = orc.reconstruct(U1, lam1)
    R0 = orc.reconstruct(U0, lam0)
    fit_explicit = 1 - np.linalg.norm(Rt - R1) / np.linalg.norm(Rt)
    assert abs(info["fit"] - fit_explicit) < 1e-10
    assert abs(info["inner"] - float(np.sum(Rt * R1))) < 1e-11 * abs(info["inner"])
    eta_explicit = np.linalg.norm(R1 - R0) / np.linalg.norm(R0)
    assert abs(orc.eta(U1, lam1, U0, lam0) - eta_explicit) < 1e-10 * eta_explicit


# ---------------------------------------------------------------- energies

def test_cp_energy_matrix_free_equals_explicit(tiny):
    U, lam, _ = orc.cp_als(tiny.Bvv, tiny.tau, tiny.factors, 3)
    E_free = orc.energy_cp(tiny.B, tiny.o, U, lam)
    E_expl = orc.energy_of_tensor(orc.reconstruct(U, lam), tiny.B, tiny.o)
    assert abs(E_free - E_expl) < 1e-13 * max(abs(E_expl), 1e-300) + 1e-18


def test_energy_invariant_under_symmetrisation(tiny):
    U, lam, _ = orc.cp_als(tiny.Bvv, tiny.tau, tiny.factors, 2)
    Rt = orc.reconstruct(U, lam)
    E1 = orc.energy_of_tensor(Rt, tiny.B, tiny.o)
    E2 = orc.energy_of_tensor(orc.symmetrise(Rt), tiny.B, tiny.o)
    assert abs(E1 - E2) < 1e-13 * abs(E1)
    # the symmetrised model is pair symmetric, the raw one is not
    S = orc.symmetrise(Rt)
    assert _rel(S, S.transpose(1, 0, 3, 2)) < 1e-15
    assert _rel(Rt, Rt.transpose(1, 0, 3, 2)) > 1e-6


def test_cp_energy_converges_to_exact_with_rank():
    inp = inputs.make_inputs(o=3, v=8, X=12, R=1, seed=0)
    n2, E_exact = orc.exact_contract(inp.B, inp.tau, inp.o)
    errs = []
    for R in (2, 8, 24, 64):
        U0 = inputs.make_factors(1, inp.o, inp.v, R)
        U, lam, hist = orc.cp_als(inp.Bvv, inp.tau, U0, 40, n2)
        errs.append(abs(orc.energy_cp(inp.B, inp.o, U, lam) - E_exact))
    assert errs[2] < 1e-2 * errs[0]
    assert errs[-1] < 1e-10 * abs(E_exact)     # rank 64 = v*v represents R exactly here


# ---------------------------------------------------------------- generator

def test_generator_deterministic_and_symmetric():
    a = inputs.make_inputs(o=4, v=6, X=9, R=5, seed=2)
    b = inputs.make_inputs(o=4, v=6, X=9, R=5, seed=2)
    assert np.array_equal(a.B, b.B) and np.array_equal(a.tau, b.tau)
    for m in orc.MODES:
        assert np.array_equal(a.factors[m], b.factors[m])
    c = inputs.make_inputs(o=4, v=6, X=9, R=5, seed=3)
    assert not np.array_equal(a.B, c.B)
    assert np.array_equal(a.B, a.B.transpose(0, 2, 1))
    assert np.max(np.abs(a.tau - a.tau.transpose(1, 0, 3, 2))) < 1e-15 * np.max(np.abs(a.tau))
    assert np.all(a.e_occ >= -1.5) and np.all(a.e_occ < -0.3)
    assert np.all(a.e_vir >= 0.1) and np.all(a.e_vir < 3.0)


def test_generator_amplitudes_follow_recipe():
    inp = inputs.make_inputs(o=3, v=4, X=5, R=2, seed=4)
    i, j, c, d = 1, 2, 3, 0
    g = float(np.dot(inp.Bov[:, i, c], inp.Bov[:, j, d]))
    den = inp.e_occ[i] + inp.e_occ[j] - inp.e_vir[c] - inp.e_vir[d]
    assert abs(inp.tau[i, j, c, d] - (g / den + inp.t1[i, c] * inp.t1[j, d])) < 1e-15


def test_generator_distribution_moments():
    z = inputs.normal(9, 0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01
    u = inputs.uniform(9, 1, 100000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.01


def test_batch_shapes_in_range():
    for o, v, X, R in inputs.batch_shapes(64, seed=0):
        assert 4 <= o <= 24 and 40 <= v <= 240 and X == 3 * v and 2 * v <= R <= 4 * v


# ---------------------------------------------------------------- stopping rules, guesses

def test_stopping_rules_fire_on_their_definitions(tiny):
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau)
    n2 = float(np.sum(Rt * Rt))
    _, _, hist, it = orc.cp_solve(tiny.Bvv, tiny.tau, tiny.factors, 60, "dfit", 1e-3, n2)
    n = len(hist)
    assert abs(hist[-1]["fit"] - hist[-2]["fit"]) < 1e-3
    assert all(abs(hist[k]["fit"] - hist[k - 1]["fit"]) >= 1e-3 for k in range(1, n - 1))
    _, _, hist, it = orc.cp_solve(tiny.Bvv, tiny.tau, tiny.factors, 60, "eta", 0.02418, n2)
    assert hist[-1]["eta"] < 0.02418 and all(h["eta"] >= 0.02418 for h in hist[:-1])
    # eta of each iterate against the previous one, from the formed tensors
    R1 = orc.reconstruct(it[-1], it[-1]["lam"])
    R0 = orc.reconstruct(it[-2], it[-2]["lam"])
    assert abs(hist[-1]["eta"] - np.linalg.norm(R1 - R0) / np.linalg.norm(R0)) < 1e-10
    _, _, hist, it = orc.cp_solve(tiny.Bvv, tiny.tau, tiny.factors, 7, "fixed")
    assert len(hist) == 7 and len(it) == 8


def test_near_optimal_cache_follows_the_offset_rule():
    guess = {m: np.full((2, 1), float(k)) for k, m in enumerate(orc.MODES)}
    pol = orc.NearOptimalGuess(guess)
    assert np.array_equal(pol.start()["b"], guess["b"])           # first CPD: random guess
    its = [{m: np.full((2, 1), 100.0 + s) for m in orc.MODES} for s in range(9)]   # n = 8 sweeps
    pol.finish(its)
    assert np.array_equal(pol.start()["a"], its[3]["a"])           # iterate n - 5 = 3
    pol.finish(its[:5])                                             # n = 4 <= 5: cache kept
    assert np.array_equal(pol.start()["j"], its[3]["j"])


def test_torch_generator_matches_numpy_generator():
    torch = pytest.importorskip("torch")
    a = inputs.make_inputs(3, 7, 5, 4, seed=13)
    B, tau, f = inputs.make_inputs_torch(3, 7, 5, 4, seed=13, device="cpu")
    assert np.max(np.abs(B.numpy() - a.B)) < 1e-14
    assert np.max(np.abs(tau.numpy() - a.tau)) < 1e-12 * np.max(np.abs(a.tau))
    for m in orc.MODES:
        assert np.array_equal(f[m], a.factors[m])


def test_torch_tau_increment_matches_numpy_across_chunks():
    torch = pytest.importorskip("torch")
    a = inputs.make_inputs(3, 5, 4, 2, seed=21)
    rms = float(np.sqrt(np.mean(a.tau ** 2)))
    for k in (1, 2):
        ref = inputs.tau_increment(a.tau, k, seed=21)
        got = inputs.tau_increment_t(torch, rms, a.tau.shape, k, seed=21, device="cpu", chunk=7)
        assert np.max(np.abs(got.numpy() - ref)) < 1e-13 * np.max(np.abs(ref))
        assert np.array_equal(got.numpy(), got.numpy().transpose(1, 0, 3, 2))   # pair symmetry



# ---------------------------------------------------------------- t1-dressed D-bar

def test_dressed_tensor_is_the_two_term_fulldfB_by_loops():
    """Eq. (fulldfB) written out term by term with loops equals R built from dress()."""
    inp = inputs.make_inputs(o=2, v=3, X=2, R=2, seed=17)
    o, v, X = 2, 3, 2
    B, t1, tau = inp.B, inp.t1, inp.tau
    R = np.zeros((v, v, o, o))
    for a, b, i, j in itertools.product(range(v), range(v), range(o), range(o)):
        s = 0.0
        for c, d, Q in itertools.product(range(v), range(v), range(X)):
            term = B[Q, o + a, o + c] * B[Q, o + b, o + d]
            for k in range(o):
                term -= 2.0 * B[Q, o + a, o + c] * B[Q, o + b, k] * t1[k, d]
            s += term * tau[i, j, c, d]
        R[a, b, i, j] = s
    Bbar = orc.dress(B, t1, o)
    assert _rel(orc.ppl_tensor(inp.Bvv, tau, Bbar), R) < 1e-13


@pytest.mark.parametrize("mode", orc.MODES)
def test_dressed_matrix_free_mttkrp_equals_explicit(tiny, mode):
    Bbar = orc.dress(tiny.B, tiny.t1, tiny.o)
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau, Bbar)
    assert _rel(orc.mttkrp(tiny.Bvv, tiny.tau, tiny.factors, mode, Bbar),
                orc.mttkrp_explicit(Rt, tiny.factors, mode)) < 1e-12


def test_dressing_moves_the_pair_symmetry_to_swapped_factors(tiny):
    Bbar = orc.dress(tiny.B, tiny.t1, tiny.o)
    R1 = orc.ppl_tensor(tiny.Bvv, tiny.tau, Bbar)          # sum B(a) Bbar(b) tau
    assert _rel(R1, R1.transpose(1, 0, 3, 2)) > 1e-3       # no longer pair symmetric
    G2 = np.einsum("Qac,Qbd->abcd", Bbar, tiny.Bvv)          # the dressing on the a side
    R2 = np.einsum("abcd,ijcd->abij", G2, tiny.tau)
    assert _rel(R1, R2.transpose(1, 0, 3, 2)) < 1e-13


def test_dressed_exact_rows_and_sweep(tiny):
    Bbar = orc.dress(tiny.B, tiny.t1, tiny.o)
    Rt = orc.ppl_tensor(tiny.Bvv, tiny.tau, Bbar)
    n2, E = orc.exact_contract(tiny.B, tiny.tau, tiny.o, Bbar)
    assert abs(n2 - float(np.sum(Rt * Rt))) < 1e-12 * n2
    assert abs(E - orc.energy_of_tensor(Rt, tiny.B, tiny.o)) < 1e-12 * abs(E)
    U1, lam1, info = orc.als_sweep(tiny.Bvv, tiny.tau, tiny.factors, np.ones(tiny.R), n2, Bbar)
    fit = 1 - np.linalg.norm(Rt - orc.reconstruct(U1, lam1)) / np.linalg.norm(Rt)
    assert abs(info["fit"] - fit) < 1e-10
