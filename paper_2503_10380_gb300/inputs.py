"""Seeded synthetic inputs for the DF particle-particle-ladder CP-ALS problem.

This module is shared by the CUDA path, its tests and the benchmark, and by
the tests of the CPU oracle.  It contains no part of the CP-ALS method: it
only draws random numbers and assembles the inputs the method consumes.

The paper's workloads are small water clusters and alkanes in DZ-F12 /
aVDZ-RI and TZ / TZ-RI basis sets (Computational details section).  Those
molecules, basis sets and integrals are not available here, so inputs are
synthetic, with the index structure and symmetries of the real ones:

* orbital energies: occupied e_i ~ U[-1.5, -0.3] Eh, virtual e_a ~ U[0.1, 3.0] Eh;
* density-fitting factor (the paper's D^{pX}_q, Eq. SQG), stored as
  B[Q, p, q] over the full orbital range n = o + v (occupied first),
  symmetric in p, q, with an auxiliary spectrum decaying as exp(-Q/15):
  B[Q] = sigma * exp(-Q/15) * (Z_Q + Z_Q^T) / sqrt(2), Z ~ N(0, 1), sigma = 0.1;
* doubles amplitudes from the DF integrals, MP2-like:
  t2[i,j,a,b] = g[i,a,j,b] / (e_i + e_j - e_a - e_b), g[iajb] = sum_Q B[Q,i,a] B[Q,j,b];
* singles t1[i,a] = 0.1 * N(0, 1) and tau = t2 + t1 x t1 (the paper's
  tau^{cd}_{ij} = t^{cd}_{ij} + t^c_i t^d_j under Eq. B), which keeps the pair
  symmetry tau[i,j,c,d] = tau[j,i,d,c];
* initial CP factors U_a, U_b (v x R) and U_i, U_j (o x R) ~ N(0, 1).

Random numbers come from a counter-based generator so that every quantity is
reproducible from (seed, stream, index) on any machine: the splitmix64
finaliser (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to a Weyl sequence, 53-bit uniforms, and
the Box-Muller transform for normals.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "uniform", "normal", "PplInputs", "make_inputs", "make_factors",
    "tau_increment", "batch_shapes", "uniform_t", "normal_t", "make_inputs_torch", "tau_increment_t",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# stream ids: each quantity draws from its own stream, so a shape change in
# one of them never shifts the numbers of another
STREAM_E_OCC, STREAM_E_VIR, STREAM_Z, STREAM_T1, STREAM_FACTORS = 0, 1, 2, 3, 4
STREAM_TAU_INCREMENT = 16  # + step index k
SIGMA_B = 0.1
DECAY_Q = 15.0
T1_SCALE = 0.1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _bits(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
                               ^ (np.uint64(stream) * _STREAM_MUL)], dtype=np.uint64))[0]
        k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(key + k * _GAMMA)


def uniform(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """`count` doubles in [0, 1) from counter positions [start, start+count)."""
    x = _bits(seed, stream, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` standard normals; normal k uses uniforms 2k and 2k+1 (Box-Muller, cos branch)."""
    u = uniform(seed, stream, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class PplInputs:
    o: int
    v: int
    X: int
    R: int
    e_occ: np.ndarray      # [o]
    e_vir: np.ndarray      # [v]
    B: np.ndarray          # [X, o+v, o+v], occupied first, symmetric in p, q
    t1: np.ndarray         # [o, v]
    tau: np.ndarray        # [o, o, v, v]
    factors: dict          # "a","b": [v, R]; "i","j": [o, R]  (initial guess)

    @property
    def Bvv(self) -> np.ndarray:
        return self.B[:, self.o:, self.o:]

    @property
    def Bov(self) -> np.ndarray:
        return self.B[:, :self.o, self.o:]


def make_factors(seed: int, o: int, v: int, R: int) -> dict:
    """Initial CP factors, filled in the order U_a, U_b, U_i, U_j (row-major)."""
    z = normal(seed, STREAM_FACTORS, 2 * v * R + 2 * o * R)
    sizes = [("a", v), ("b", v), ("i", o), ("j", o)]
    out, pos = {}, 0
    for name, dim in sizes:
        out[name] = z[pos:pos + dim * R].reshape(dim, R).copy()
        pos += dim * R
    return out


def make_inputs(o: int, v: int, X: int, R: int, seed: int = 0) -> PplInputs:
    n = o + v
    e_occ = -1.5 + 1.2 * uniform(seed, STREAM_E_OCC, o)
    e_vir = 0.1 + 2.9 * uniform(seed, STREAM_E_VIR, v)
    Z = normal(seed, STREAM_Z, X * n * n).reshape(X, n, n)
    scale = SIGMA_B * np.exp(-np.arange(X, dtype=np.float64) / DECAY_Q) / math.sqrt(2.0)
    B = (Z + Z.transpose(0, 2, 1)) * scale[:, None, None]
    del Z
    Bov = B[:, :o, o:].reshape(X, o * v)
    g = (Bov.T @ Bov).reshape(o, v, o, v)                 # g[i,a,j,b]
    denom = (e_occ[:, None, None, None] + e_occ[None, None, :, None]
             - e_vir[None, :, None, None] - e_vir[None, None, None, :])
    t2 = (g / denom).transpose(0, 2, 1, 3)                # t2[i,j,a,b]
    t1 = T1_SCALE * normal(seed, STREAM_T1, o * v).reshape(o, v)
    tau = np.ascontiguousarray(t2 + t1[:, None, :, None] * t1[None, :, None, :])
    return PplInputs(o, v, X, R, e_occ, e_vir, np.ascontiguousarray(B), t1, tau,
                     make_factors(seed, o, v, R))


def tau_increment(tau0: np.ndarray, k: int, seed: int = 0) -> np.ndarray:
    """Increment for step k of a CC-like sequence tau_k = tau_{k-1} + dtau_k.

    dtau_k = 0.3**k * rms(tau_0) * (Z + Z^pair) / sqrt(2), Z ~ N(0,1), where
    Z^pair[i,j,c,d] = Z[j,i,d,c]; it keeps the pair symmetry of tau.
    """
    o, _, v, _ = tau0.shape
    Z = normal(seed, STREAM_TAU_INCREMENT + k, tau0.size).reshape(tau0.shape)
    Zs = (Z + Z.transpose(1, 0, 3, 2)) / math.sqrt(2.0)
    rms = math.sqrt(float(np.mean(tau0 * tau0)))
    return (0.3 ** k) * rms * Zs


def batch_shapes(count: int, seed: int = 0):
    """Uneven instance shapes: o in [4,24], v in [40,240], X = 3v, R in [2v, 4v]."""
    u = uniform(seed, 64, 3 * count).reshape(count, 3)
    shapes = []
    for k in range(count):
        o = 4 + int(u[k, 0] * 21)
        v = 40 + int(u[k, 1] * 201)
        R = 2 * v + int(u[k, 2] * (2 * v + 1))
        shapes.append((o, v, 3 * v, R))
    return shapes


# --------------------------------------------------------------------------
# the same generator in torch (for large sizes, on the device)
# --------------------------------------------------------------------------

def _i64(x: int) -> int:
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(torch, z, k: int):
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64_t(torch, z):
    z = (z ^ _lsr(torch, z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _lsr(torch, z, 27)) * _i64(0x94D049BB133111EB)
    return z ^ _lsr(torch, z, 31)


def uniform_t(torch, seed: int, stream: int, count: int, device, start: int = 0):
    with np.errstate(over="ignore"):
        key = int(_mix64(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (np.uint64(stream) * _STREAM_MUL)],
                                  dtype=np.uint64))[0])
    k = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    x = _mix64_t(torch, _i64(key) + k * _i64(int(_GAMMA)))
    return _lsr(torch, x, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def normal_t(torch, seed: int, stream: int, count: int, device, start: int = 0):
    """Normals start .. start+count-1 of the stream (normal k uses uniforms 2k, 2k+1)."""
    u = uniform_t(torch, seed, stream, 2 * count, device, start=2 * start)
    u1, u2 = u[0::2], u[1::2]
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)


def make_inputs_torch(o: int, v: int, X: int, R: int, seed: int = 0, device="cuda"):
    """make_inputs with torch on `device`: returns (B, tau, factors) with B, tau
    FP64 tensors on the device and the factors as numpy arrays.  Same recipe and
    counter streams as make_inputs (values agree to rounding of log/cos and of
    the sum over Q)."""
    import torch
    n = o + v
    e_occ = -1.5 + 1.2 * uniform_t(torch, seed, STREAM_E_OCC, o, device)
    e_vir = 0.1 + 2.9 * uniform_t(torch, seed, STREAM_E_VIR, v, device)
    B = normal_t(torch, seed, STREAM_Z, X * n * n, device).view(X, n, n)
    scale = SIGMA_B * torch.exp(-torch.arange(X, dtype=torch.float64, device=device) / DECAY_Q) / math.sqrt(2.0)
    B = (B + B.transpose(1, 2)) * scale[:, None, None]
    Bov = B[:, :o, o:].reshape(X, o * v)
    g = (Bov.T @ Bov).view(o, v, o, v)
    denom = (e_occ[:, None, None, None] + e_occ[None, None, :, None]
             - e_vir[None, :, None, None] - e_vir[None, None, None, :])
    tau = (g / denom).permute(0, 2, 1, 3).contiguous()
    del g, denom
    t1 = T1_SCALE * normal_t(torch, seed, STREAM_T1, o * v, device).view(o, v)
    tau += t1[:, None, :, None] * t1[None, :, None, :]
    return B.contiguous(), tau, make_factors(seed, o, v, R)


def tau_increment_t(torch, tau0_rms: float, shape, k: int, seed: int = 0, device="cuda", chunk: int = 1 << 26):
    """tau_increment on `device`, given rms(tau_0); the normals are drawn in
    chunks of `chunk` so that the counter tensors stay small."""
    n = 1
    for d in shape:
        n *= d
    Z = torch.empty(n, dtype=torch.float64, device=device)
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        Z[s:s + c] = normal_t(torch, seed, STREAM_TAU_INCREMENT + k, c, device, start=s)
    Z = Z.view(*shape)
    out = Z + Z.permute(1, 0, 3, 2)
    out *= (0.3 ** k) * tau0_rms / math.sqrt(2.0)
    return out
