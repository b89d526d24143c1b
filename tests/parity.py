"""Element-wise comparison of the CUDA path with the CPU oracle.

Two checks per compared array, each reporting the worst element on failure:

1. A bound from absolute values.  For a result that is a chain of products
   and sums (an MTTKRP, the formed tensor), evaluating the same chain on the
   absolute values of every input gives, per element, the sum of |terms|; the
   error of any evaluation order in a floating-point format with per-product
   relative error p and accumulation error q per addition is at most
   (p + q) times that sum, per contraction of the chain.  gamma below is that
   bound for each precision (derivations beside the constants).

2. A bound per column of the reference: every element of column r (one rank
   component, one r-chunk position) must be within tol times the largest
   |reference| of that column.  The signed sums of these chains cancel heavily
   (the absolute-value chain exceeds the result by orders of magnitude), so (1)
   alone would pass a wrong column; (2) catches a bad column, a bad r-chunk or a
   wrong ragged tail of rows, whose errors are of the size of the column itself.
"""

from __future__ import annotations

import numpy as np

# (1) per-element bound factor for one MTTKRP (a chain of four contractions,
# the last one split over K and reduced in FP64), in units of the
# absolute-value chain:
#   fp64   4 contractions of K <= 1.1e6 with u = 2^-53 on both sides: <= 1e-9
#   tf32x3 per contraction 3*2^-22 (dropped lo*lo and the split remainders)
#          + 2^-22 (the next operand's hi/lo split) + 12*2^-23 (round toward
#          zero inside one restarted K block of 12 MMAs) + n_c*2^-24 (FP32 sums
#          of n_c K blocks, n_c <= 2280 for the longest split-K slice): <= 2e-4
#   bf16x3 per contraction 3*2^-16 + 2^-16, accumulation without restarts:
#          one ulp per MMA over <= 14000 MMAs of a split-K slice (1.7e-3): <= 3e-3
#   tf32   per contraction 2*2^-11 + 2^-11, accumulation as bf16x3: <= 1e-2
GAMMA = {"fp64": 1e-9, "tf32x3": 2e-4, "bf16x3": 3e-3, "tf32": 1e-2}

# (2) per-column bound for one MTTKRP (the largest normwise relative error
# measured on GB300 over the test shapes and the benchmark sizes was 4.1e-15,
# 1.5e-6, 3.9e-5 and 9.6e-4; a column's worst element relative to the
# column's largest entry is of the same order)
COLTOL = {"fp64": 1e-12, "tf32x3": 1e-5, "bf16x3": 5e-4, "tf32": 1e-2}


def _where(r, shape):
    i = int(np.argmax(r))
    return tuple(int(x) for x in np.unravel_index(i, shape))


def check_abs_bound(got, ref, ref_abs, gamma, what=""):
    """|got - ref| <= gamma * ref_abs + tiny, element by element."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape == np.shape(ref_abs), (what, got.shape, ref.shape, np.shape(ref_abs))
    err = np.abs(got - ref)
    bound = gamma * np.asarray(ref_abs) + 1e-300
    r = err / bound
    if not np.all(r <= 1.0):
        w = _where(r, r.shape)
        raise AssertionError(f"{what}: element {w} got {got[w]!r} ref {ref[w]!r} |err| {err[w]:.3e} exceeds "
                             f"{gamma:g} x |chain| = {bound[w]:.3e} (ratio {r[w]:.3g})")
    return float(np.max(err / (np.asarray(ref_abs) + 1e-300)))


def check_columns(got, ref, tol, what="", axis=0):
    """Every element within tol x (largest |ref| of its column), columns along
    the last axis for 2-D arrays (axis = the reduced row axis)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = np.abs(got - ref)
    scale = np.max(np.abs(ref), axis=axis, keepdims=True)
    r = err / (tol * scale + 1e-300)
    if not np.all(r <= 1.0):
        w = _where(r, r.shape)
        col = w[1] if len(w) > 1 else 0
        raise AssertionError(f"{what}: element {w} (column {col}) got {got[w]!r} ref {ref[w]!r} |err| "
                             f"{err[w]:.3e} exceeds {tol:g} x column max {float(np.broadcast_to(scale, r.shape)[w]):.3e}")
    return float(np.max(err / (scale + 1e-300)))


def abs_factors(U: dict) -> dict:
    return {k: np.abs(v) for k, v in U.items()}


def check_mttkrp(got, ref, ref_abs, prec, what=""):
    """Both element-wise checks for one MTTKRP [dim][R]."""
    check_abs_bound(got, ref, ref_abs, GAMMA[prec], what + " (abs-chain bound)")
    check_columns(got, ref, COLTOL[prec], what + " (per-column bound)")
