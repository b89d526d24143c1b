"""Plain FP64 CPU oracle for matrix-free CP-ALS of the DF particle-particle ladder.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import or call this module.  It shares no
code with the CUDA path and imports nothing from it.

What it computes (paper: Pierce, "Towards Using Matrix-Free Tensor
Decompositions to Systematically Improve Approximate Tensor-Networks"):

* the DF particle-particle-ladder tensor, Eq. (dfB) with D-bar = D,
      R[a,b,i,j] = sum_{Q,c,d} B[Q,a,c] B[Q,b,d] tau[i,j,c,d],
  or with the t1-dressed D-bar of Eq. (fulldfB) on the b side, formed
  explicitly only at tiny sizes;
* its rank-R CP model, Eq. (cp-ppl): R~[a,b,i,j] = sum_r lam_r Ua[a,r] Ub[b,r] Ui[i,r] Uj[j,r]
  (paper's alpha, beta, gamma, rho; unit-norm columns with the scales in lam,
  The Canonical Polyadic Decomposition section);
* the matrix-free MTTKRP of each mode, Eqs. (full_der), (distribute),
  (foreachr) and the cached intermediates listed with them and in Table
  (table:scaling);
* the ALS update, Optimizing the CP-PPL tensor-network section: W (here V) as
  the Hadamard product of the three other Gram matrices, a Cholesky solve of
  the normal equations, column normalisation;
* the fit, Eq. (cpfit) through the residual expansion and Eq. (cp_norm2), and
  the eta criterion, Eqs. (N3_stopping) and (new_conv);
* the PPL energy E = sum R[abij] (2 g[iajb] - g[ibja]) for the exact tensor and
  for the CP model (explicitly and matrix-free).

Readings where the paper is silent (each also listed in the design notes):
* modes b, i, j: the paper derives the update for alpha only and says the
  others follow the same way; their MTTKRPs are derived here from Eq. (dfB);
* Gauss-Seidel mode order a, b, i, j, each update using the newest factors;
* the solve is a Cholesky factorisation in which a pivot that is not larger
  than tol = max(2^-52 * R * max_k V_kk, 1e-300) is replaced by tol (counted),
  then two triangular solves; this is the reading of "a symmetric, square
  linear solve algorithm such as the Cholesky decomposition" for a
  semidefinite V;
* a zero column after the solve keeps lam_r = 0 and is left unscaled.

Everything here is FP64 numpy.  Library primitives (matmul, tensordot,
einsum, triangular solves) serve as single steps; nothing is blocked, fused
or reordered beyond what the equations state.

Parity pins live in tests/test_oracle_pins.py.  Unpinned: nothing in the
ALS step chain; the paper prints no numeric example, so pins are brute force
on tiny inputs, closed forms, invariants and special cases.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_triangular

MODES = ("a", "b", "i", "j")


# --------------------------------------------------------------------------
# explicit tensors (tiny sizes only)
# --------------------------------------------------------------------------

def dress(B: np.ndarray, t1: np.ndarray, o: int) -> np.ndarray:
    """D-bar^{bX}_d = D^{bX}_d - 2 sum_k D^{bX}_k t^k_d, the intermediate defined after
    Eq. (fulldfB) (its X index, missing in the printed definition, restored).
    B [X][o+v][o+v], t1 [o][v] (t^a_i as t1[i, a]).  Returns D-bar over (Q, b, d) = [X][v][v]."""
    Bvv = B[:, o:, o:]
    Bvo = B[:, o:, :o]
    return Bvv - 2.0 * np.einsum("Qbk,kd->Qbd", Bvo, t1)


def ppl_tensor(Bvv: np.ndarray, tau: np.ndarray, Bbar: np.ndarray | None = None) -> np.ndarray:
    """R[a,b,i,j] = sum_cd (sum_Q B[Q,a,c] Bbar[Q,b,d]) tau[i,j,c,d]; Eq. (dfB), with
    Bbar = B unless a dressed D-bar is given."""
    Bb = Bvv if Bbar is None else Bbar
    G = np.einsum("Qac,Qbd->abcd", Bvv, Bb)
    return np.einsum("abcd,ijcd->abij", G, tau)


def reconstruct(U: dict, lam: np.ndarray) -> np.ndarray:
    """CP model of Eq. (cp-ppl) with the column scales lam restored."""
    return np.einsum("r,ar,br,ir,jr->abij", lam, U["a"], U["b"], U["i"], U["j"])


def symmetrise(Rt: np.ndarray) -> np.ndarray:
    """0.5 (R~[a,b,i,j] + R~[b,a,j,i]), the post-reconstruction symmetrisation of the CPD-PPL section."""
    return 0.5 * (Rt + Rt.transpose(1, 0, 3, 2))


def mttkrp_explicit(Rt: np.ndarray, U: dict, mode: str) -> np.ndarray:
    """MTTKRP of a formed 4-way tensor: the sum over the other three indices
    of R times the other three factors (the first term of the gradient in the
    Optimizing the CP-PPL tensor-network section)."""
    spec = {
        "a": "abij,br,ir,jr->ar",
        "b": "abij,ar,ir,jr->br",
        "i": "abij,ar,br,jr->ir",
        "j": "abij,ar,br,ir->jr",
    }[mode]
    others = [U[m] for m in MODES if m != mode]
    return np.einsum(spec, Rt, *others, optimize=True)


# --------------------------------------------------------------------------
# matrix-free MTTKRP
# --------------------------------------------------------------------------

def tau_r(tau: np.ndarray, Ui: np.ndarray, Uj: np.ndarray) -> np.ndarray:
    """tau^{cd}_r = sum_ij gamma^r_i rho^r_j tau^{cd}_ij (first row of Table (table:scaling)).

    The Khatri-Rao product KR[ij, r] = Ui[i,r] Uj[j,r] is formed and
    contracted with tau by one matrix product.  Returns [R, v(c), v(d)].
    """
    o, _, v, _ = tau.shape
    KR = (Ui[:, None, :] * Uj[None, :, :]).reshape(o * o, -1)
    T = tau.reshape(o * o, v * v).T @ KR            # [cd, r]
    return np.ascontiguousarray(T.T).reshape(-1, v, v)


def dbar_r(Bvv: np.ndarray, U: np.ndarray) -> np.ndarray:
    """D-bar^{rX}_d = sum_b D^{bX}_d U[b, r] (second row of Table (table:scaling)).

    Contracts the first orbital index of B[Q, b, d] with U.  Returns [R, X, v].
    """
    return np.tensordot(U, Bvv, axes=([0], [1]))      # [r, Q, d]


def compound_view(Bvv):
    """D^{aQ}_c as a v x (X v) matrix over the compound index {Q c} (Eq. foreachr)."""
    X, v, _ = Bvv.shape
    return np.ascontiguousarray(Bvv.transpose(1, 0, 2)).reshape(v, X * v)


def mttkrp_a(Bvv, T, Db):
    """Mode a (alpha), Eqs. (distribute) and (foreachr): for each r, the gemm
    inner[Q, c] = sum_d Db[r, Q, d] T[r, c, d], then the gemv over the
    compound index {Q c} with D^{aQ}_c."""
    Bc = compound_view(Bvv)
    R = T.shape[0]
    M = np.zeros((Bc.shape[0], R))
    for r in range(R):
        inner = Db[r] @ T[r].T                           # [Q, c]
        M[:, r] = Bc @ inner.reshape(-1)
    return M


def mttkrp_b(Bvv, T, Da):
    """Mode b (beta), the same chain with the roles of (a, c) and (b, d)
    exchanged: inner[Q, d] = sum_c Da[r, Q, c] T[r, c, d], then
    M[b, r] = sum_{Q d} B[Q, b, d] inner[Q, d]."""
    Bc = compound_view(Bvv)
    R = T.shape[0]
    M = np.zeros((Bc.shape[0], R))
    for r in range(R):
        inner = Da[r] @ T[r]                             # [Q, d]
        M[:, r] = Bc @ inner.reshape(-1)
    return M


def p_intermediate(Bvv, tau, Ua, Ub, Bbar=None):
    """For modes i and j: S_r[c, d] = sum_Q Da[r,Q,c] Db[r,Q,d] and
    P[i, j, r] = sum_cd tau[i,j,c,d] S_r[c,d]; Db from D-bar when dressed."""
    o, _, v, _ = tau.shape
    Da = dbar_r(Bvv, Ua)
    Db = dbar_r(Bvv if Bbar is None else Bbar, Ub)
    R = Ua.shape[1]
    S = np.empty((R, v, v))
    for r in range(R):
        S[r] = Da[r].T @ Db[r]
    P = tau.reshape(o * o, v * v) @ S.reshape(R, v * v).T
    return P.reshape(o, o, R)


def mttkrp(Bvv: np.ndarray, tau: np.ndarray, U: dict, mode: str, Bbar=None) -> np.ndarray:
    """Matrix-free MTTKRP of R (never formed) for one mode; result [dim, R].  With a
    dressed D-bar, the b side (second factor of Eq. dfB) uses it."""
    Bb = Bvv if Bbar is None else Bbar
    if mode == "a":
        return mttkrp_a(Bvv, tau_r(tau, U["i"], U["j"]), dbar_r(Bb, U["b"]))
    if mode == "b":
        return mttkrp_b(Bb, tau_r(tau, U["i"], U["j"]), dbar_r(Bvv, U["a"]))
    P = p_intermediate(Bvv, tau, U["a"], U["b"], Bbar)
    if mode == "i":
        return np.einsum("ijr,jr->ir", P, U["j"])
    if mode == "j":
        return np.einsum("ijr,ir->jr", P, U["i"])
    raise ValueError(mode)


# --------------------------------------------------------------------------
# normal equations
# --------------------------------------------------------------------------

def gram(U: np.ndarray) -> np.ndarray:
    return U.T @ U


def hadamard_v(U: dict, mode: str) -> np.ndarray:
    """W of the Optimizing the CP-PPL section: the elementwise product of the
    Gram matrices of the three factors that are held fixed."""
    V = None
    for m in MODES:
        if m == mode:
            continue
        G = gram(U[m])
        V = G if V is None else V * G
    return V


def cholesky_clamped(V: np.ndarray):
    """Lower Cholesky factor of V, column by column; a pivot not above
    tol = max(2^-52 R max_k V_kk, 1e-300) is replaced by tol.  Returns (L, nclamped)."""
    R = V.shape[0]
    tol = max(2.0 ** -52 * R * float(np.max(np.diag(V))) if R else 0.0, 1e-300)
    L = np.zeros_like(V)
    nclamp = 0
    for j in range(R):
        d = V[j, j] - L[j, :j] @ L[j, :j]
        if not d > tol:
            d = tol
            nclamp += 1
        L[j, j] = math.sqrt(d)
        if j + 1 < R:
            L[j + 1:, j] = (V[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L, nclamp


def solve_normal(M: np.ndarray, V: np.ndarray):
    """U~ = M V^{-1} through V = L L^T: Z = M L^{-T}, then U~ = Z L^{-1}.
    Returns (U~, nclamped)."""
    L, nclamp = cholesky_clamped(V)
    Zt = solve_triangular(L, M.T, lower=True)          # L Z^T = M^T
    Ut = solve_triangular(L.T, Zt, lower=False)        # L^T U~^T = Z^T
    return Ut.T, nclamp


def normalise(Ut: np.ndarray):
    """Unit 2-norm columns with the norms returned as lam; a zero column keeps lam = 0."""
    lam = np.sqrt(np.sum(Ut * Ut, axis=0))
    U = Ut.copy()
    nz = lam > 0
    U[:, nz] /= lam[nz]
    return U, lam


# --------------------------------------------------------------------------
# fit, eta, norms
# --------------------------------------------------------------------------

def cp_norm2(U: dict, lam: np.ndarray) -> float:
    """||R~||^2 = lam^T (Ua^T Ua * Ub^T Ub * Ui^T Ui * Uj^T Uj) lam; Eq. (cp_norm2)."""
    H = gram(U["a"]) * gram(U["b"]) * gram(U["i"]) * gram(U["j"])
    return float(lam @ H @ lam)


def cp_cross(U1: dict, lam1: np.ndarray, U0: dict, lam0: np.ndarray) -> float:
    """<R~_1, R~_0> = lam1^T (prod_m U1_m^T U0_m) lam0, the middle term of Eq. (new_conv)."""
    H = np.ones((lam1.size, lam0.size))
    for m in MODES:
        H = H * (U1[m].T @ U0[m])
    return float(lam1 @ H @ lam0)


def eta(U1, lam1, U0, lam0) -> float:
    """eta = ||R~_n - R~_{n-1}|| / ||R~_{n-1}||; Eqs. (N3_stopping), (new_conv)."""
    n1 = cp_norm2(U1, lam1)
    n0 = cp_norm2(U0, lam0)
    num2 = n1 - 2.0 * cp_cross(U1, lam1, U0, lam0) + n0
    return math.sqrt(max(num2, 0.0)) / math.sqrt(n0)


def inner_from_mttkrp(M_last: np.ndarray, U_last: np.ndarray, lam: np.ndarray) -> float:
    """<R, R~> = sum_r lam_r sum_x M[x, r] U[x, r], the cross term of the residual
    expansion under Eq. (cpfit), taken from the last mode's MTTKRP."""
    return float(np.sum(lam * np.sum(M_last * U_last, axis=0)))


def fit_value(normR2: float, inner: float, norm2: float) -> float:
    """Delta = 1 - ||R - R~|| / ||R||, Eq. (cpfit), with
    ||R - R~||^2 = ||R||^2 - 2 <R, R~> + ||R~||^2."""
    return 1.0 - math.sqrt(max(normR2 - 2.0 * inner + norm2, 0.0)) / math.sqrt(normR2)


# --------------------------------------------------------------------------
# ALS
# --------------------------------------------------------------------------

def als_sweep(Bvv, tau, U: dict, lam: np.ndarray, normR2: float | None = None, Bbar=None):
    """One ALS sweep a -> b -> i -> j.  tau_r is shared by modes a and b and
    P by modes i and j (the cached intermediates of the paper).  Returns
    (U, lam, info) with info = dict(inner, norm2, fit, nclamped, M)."""
    U = {m: U[m].copy() for m in MODES}
    Bb = Bvv if Bbar is None else Bbar
    nclamp = 0
    Ms = {}
    T = tau_r(tau, U["i"], U["j"])
    for mode in ("a", "b"):
        if mode == "a":
            M = mttkrp_a(Bvv, T, dbar_r(Bb, U["b"]))
        else:
            M = mttkrp_b(Bb, T, dbar_r(Bvv, U["a"]))
        Ut, nc = solve_normal(M, hadamard_v(U, mode))
        U[mode], lam = normalise(Ut)
        Ms[mode] = M
        nclamp += nc
    P = p_intermediate(Bvv, tau, U["a"], U["b"], Bbar)
    for mode in ("i", "j"):
        if mode == "i":
            M = np.einsum("ijr,jr->ir", P, U["j"])
        else:
            M = np.einsum("ijr,ir->jr", P, U["i"])
        Ut, nc = solve_normal(M, hadamard_v(U, mode))
        U[mode], lam = normalise(Ut)
        Ms[mode] = M
        nclamp += nc
    inner = inner_from_mttkrp(Ms["j"], U["j"], lam)
    norm2 = cp_norm2(U, lam)
    fit = fit_value(normR2, inner, norm2) if normR2 else None
    return U, lam, dict(inner=inner, norm2=norm2, fit=fit, nclamped=nclamp, M=Ms)


def cp_als(Bvv, tau, U0: dict, nsweeps: int, normR2: float | None = None, lam0=None, Bbar=None):
    """nsweeps ALS sweeps from the initial factors U0 (lam starts at ones).
    Returns (U, lam, history) with one info dict per sweep (plus eta)."""
    U = {m: np.array(U0[m], dtype=np.float64, copy=True) for m in MODES}
    lam = np.ones(U["a"].shape[1]) if lam0 is None else np.array(lam0, dtype=np.float64)
    hist = []
    for _ in range(nsweeps):
        Un, lamn, info = als_sweep(Bvv, tau, U, lam, normR2, Bbar)
        info["eta"] = eta(Un, lamn, U, lam)
        hist.append(info)
        U, lam = Un, lamn
    return U, lam, hist


# --------------------------------------------------------------------------
# energies and the exact contraction
# --------------------------------------------------------------------------

def g_ovov(B: np.ndarray, o: int) -> np.ndarray:
    """g[i,a,j,b] = sum_Q B[Q,i,a] B[Q,j,b]; Eq. (SQG)."""
    Bov = B[:, :o, o:]
    return np.einsum("Qia,Qjb->iajb", Bov, Bov)


def energy_of_tensor(Rt: np.ndarray, B: np.ndarray, o: int) -> float:
    """E = sum_{abij} R[a,b,i,j] (2 g[iajb] - g[ibja]) in Eh."""
    g = g_ovov(B, o)
    L = 2.0 * g.transpose(1, 3, 0, 2) - g.transpose(3, 1, 0, 2)   # [a,b,i,j]
    return float(np.sum(Rt * L))


def energy_cp(B: np.ndarray, o: int, U: dict, lam: np.ndarray) -> float:
    """CP energy without forming R~:
    E = sum_r lam_r sum_Q [2 A_Q(Ui,Ua) A_Q(Uj,Ub) - A_Q(Ui,Ub) A_Q(Uj,Ua)],
    A_Q(x, y)_r = sum_{i,a} B[Q,i,a] x[i,r] y[a,r]."""
    Bov = B[:, :o, o:]

    def A(x, y):
        return np.einsum("Qia,ir,ar->Qr", Bov, x, y, optimize=True)

    t = 2.0 * A(U["i"], U["a"]) * A(U["j"], U["b"]) - A(U["i"], U["b"]) * A(U["j"], U["a"])
    return float(np.sum(lam * np.sum(t, axis=0)))


def exact_rows(B: np.ndarray, tau: np.ndarray, o: int, a_rows, Bbar=None) -> tuple:
    """Rows R[a, :, :, :] of the exact tensor for the given a, with their
    contributions to ||R||^2 and to E.  Returns (R_rows [len, v, o, o], norm2_part, E_part)."""
    Bvv = B[:, o:, o:]
    Bb = Bvv if Bbar is None else Bbar
    Bov = B[:, :o, o:]
    v = Bvv.shape[1]
    tau2 = tau.reshape(o * o, v * v)
    rows, n2, E = [], 0.0, 0.0
    for a in a_rows:
        Ga = np.tensordot(Bvv[:, a, :], Bb, axes=([0], [0]))         # [c, b, d]
        Ra = (Ga.transpose(1, 0, 2).reshape(v, v * v) @ tau2.T).reshape(v, o, o)   # [b, i, j]
        # 2 g[i a j b] - g[i b j a]
        g1 = np.einsum("Qi,Qjb->bij", Bov[:, :, a], Bov)
        g2 = np.einsum("Qib,Qj->bij", Bov, Bov[:, :, a])
        rows.append(Ra)
        n2 += float(np.sum(Ra * Ra))
        E += float(np.sum(Ra * (2.0 * g1 - g2)))
    return np.stack(rows) if rows else np.zeros((0, v, o, o)), n2, E


def exact_contract(B: np.ndarray, tau: np.ndarray, o: int, Bbar=None):
    """||R||^2 and E_exact over all rows a."""
    v = B.shape[1] - o
    _, n2, E = exact_rows(B, tau, o, range(v), Bbar)
    return n2, E


# --------------------------------------------------------------------------
# stopping rules and initial-guess policies
# --------------------------------------------------------------------------

def cp_solve(Bvv, tau, U0: dict, max_sweeps: int, rule: str = "fixed", eps: float = 0.0,
             normR2: float | None = None, lam0=None):
    """ALS sweeps until a stopping rule fires (Low cost CPD stopping condition section).

    rule "fixed": exactly max_sweeps sweeps.
    rule "dfit":  stop after sweep n >= 2 when |Delta_n - Delta_{n-1}| < eps, Delta the fit of
                  Eq. (cpfit) (Eq. canon, read with an absolute value); needs normR2.
    rule "eta":   stop after sweep n >= 1 when eta_n < eps, Eq. (N3_stopping), eta_1 measured
                  against the initial guess.
    Returns (U, lam, hist, iterates) where iterates[k] are the factors after sweep k
    (iterates[0] = the start), as dicts including "lam"."""
    U = {m: np.array(U0[m], dtype=np.float64, copy=True) for m in MODES}
    lam = np.ones(U["a"].shape[1]) if lam0 is None else np.array(lam0, dtype=np.float64)
    iterates = [dict(U, lam=lam.copy())]
    hist = []
    for n in range(1, max_sweeps + 1):
        Un, lamn, info = als_sweep(Bvv, tau, U, lam, normR2)
        info["eta"] = eta(Un, lamn, U, lam)
        hist.append(info)
        U, lam = Un, lamn
        iterates.append(dict(U, lam=lam.copy()))
        if rule == "dfit" and n >= 2 and abs(hist[-1]["fit"] - hist[-2]["fit"]) < eps:
            break
        if rule == "eta" and info["eta"] < eps:
            break
    return U, lam, hist, iterates


class NearOptimalGuess:
    """The "Near-Optimal guess" of the Role of the Initial Guess section: when a CPD needs
    n > 5 ALS iterations, the factors after iteration n - 5 are cached; otherwise the
    previous cache is kept.  Every CPD after the first starts from the cache; the first
    (and any CPD while no cache exists yet) starts from the random guess."""

    OFFSET = 5

    def __init__(self, random_guess: dict):
        self.random_guess = {m: np.array(random_guess[m], copy=True) for m in MODES}
        self.cache = None

    def start(self) -> dict:
        src = self.cache if self.cache is not None else self.random_guess
        return {m: src[m].copy() for m in MODES}

    def finish(self, iterates: list):
        n = len(iterates) - 1
        if n > self.OFFSET:
            self.cache = {m: iterates[n - self.OFFSET][m].copy() for m in MODES}
