"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Sizes span several tiles and ragged tails.  Tolerances:
* FP64 form: 1e-12 relative for one MTTKRP (a few hundred FP64 roundings of
  O(1) terms), 1e-8 after several ALS sweeps (Cholesky solves amplify
  rounding by the condition number of V).
* BF16X3: each operand is split into bf16 hi + lo with |x - hi - lo| <= 2^-16 |x|;
  dropping lo*lo leaves <= 3 * 2^-16 relative per product, FP32 accumulation
  adds K * 2^-24.  The MTTKRP chains four contractions, so the normwise
  bound is about 4 * (3 * 2^-16) ~ 2e-4; the tests use 1e-4 normwise
  (errors add in quadrature in practice).
* TF32: operands rounded to nearest with 10 explicit bits, |dx| <= 2^-11 |x|,
  i.e. about 2 * 2^-11 = 1e-3 per product and 4e-3 for the chain; tests use 4e-3.
* TF32X3: hi = tf32(x), lo = tf32(x - hi), |x - hi - lo| <= 2^-22 |x|; with lo*lo
  dropped, <= 3 * 2^-22 relative per product; the accumulator is restarted every
  32 K elements and the chunks are added with round-to-nearest, so the
  tensor core's round-toward-zero accumulation adds at most one ulp per MMA of
  one chunk.  Chain bound about 4 * 3 * 2^-22 + 4 * 16 * 2^-23 ~ 1e-5.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ppl_oracle as orc
from paper_2503_10380_gb300 import binding, inputs
from parity import COLTOL, GAMMA, abs_factors, check_abs_bound, check_columns, check_mttkrp

pytestmark = pytest.mark.gpu

TOL_MTTKRP = {"fp64": 1e-12, "bf16x3": 1e-4, "tf32": 4e-3, "tf32x3": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _mttkrp_refs(Bvv, tau, U, Bbar=None):
    """Oracle MTTKRP of every mode and the same chains on absolute values."""
    aB, aT, aU = np.abs(Bvv), np.abs(tau), abs_factors(U)
    aBb = None if Bbar is None else np.abs(Bbar)
    refs = {m: orc.mttkrp(Bvv, tau, U, m, Bbar) for m in orc.MODES}
    abss = {m: orc.mttkrp(aB, aT, aU, m, aBb) for m in orc.MODES}
    return refs, abss


def _factors(cp):
    return {k: t.cpu().numpy().copy() for k, t in cp.factors().items()}


def _check_factors(f, U_ref, lam_ref, tol, what):
    """Every factor column by column, and lam element by element, against the oracle."""
    for m in orc.MODES:
        check_columns(f[m], U_ref[m], tol, f"{what} U_{m}")
    check_columns(f["lam"][None, :], lam_ref[None, :], tol, f"{what} lam", axis=None)


SHAPES = [
    (5, 24, 72, 48),     # config 0
    (3, 13, 17, 19),     # every extent ragged
    (1, 9, 5, 1),        # o = 1, R = 1
    (7, 40, 90, 150),    # several tiles, ragged tails
]


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "tf32x3"])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 600, 200), (37, 130, 1000), (300, 16, 24)])
def test_tc_gemm_building_block(prec, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    C = binding.tc_gemm(_dev(A), _dev(B), prec).cpu().numpy()
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    bound = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    tol = {"bf16x3": 3 * 2.0 ** -16 + K * 2.0 ** -23, "tf32": 2 * 2.0 ** -11 + K * 2.0 ** -23,
           "tf32x3": 3 * 2.0 ** -22 + K * 2.0 ** -23}[prec]
    assert np.all(np.abs(C - ref) <= tol * bound + 1e-30)


def test_restarted_accumulation_has_no_drift():
    """Operands exact in tf32 and all products positive: every rounding of the
    sum goes the same way.  The tcgen05 FP32 accumulator rounds toward zero at
    each MMA, so one accumulator over K = 8192 loses about half an ulp per MMA;
    TF32X3 restarts it every 32 K elements and adds the chunks with
    round-to-nearest, so only the few MMAs inside one chunk still round down
    (about 2e-7 relative here, against about 4e-5 for one accumulator)."""
    g = torch.Generator().manual_seed(5)
    M, N, K = 256, 192, 8192
    A = torch.randint(1024, 2048, (M, K), generator=g).float() / 2048
    B = torch.randint(1024, 2048, (N, K), generator=g).float() / 2048
    ref = A.double() @ B.double().T
    C = binding.tc_gemm(A.cuda(), B.cuda(), "tf32x3").double().cpu()
    drift = float(((C - ref) * torch.sign(ref)).sum() / ref.abs().sum())
    assert abs(drift) < 1e-6, drift
    C1 = binding.tc_gemm(A.cuda(), B.cuda(), "tf32").double().cpu()
    drift1 = float(((C1 - ref) * torch.sign(ref)).sum() / ref.abs().sum())
    assert drift1 <= 0.0          # one unrestarted accumulator never rounds up


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32", "tf32x3"])
@pytest.mark.parametrize("shape", SHAPES)
def test_mttkrp_each_mode(prec, shape):
    o, v, X, R = shape
    inp = inputs.make_inputs(o, v, X, R, seed=1)
    refs, abss = _mttkrp_refs(inp.Bvv, inp.tau, inp.factors)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec)
    for m in orc.MODES:
        M = cp.mttkrp(m).cpu().numpy()
        check_mttkrp(M, refs[m], abss[m], prec, f"{prec} {shape} mode {m}")
        assert _rel(M, refs[m]) < TOL_MTTKRP[prec], (m, _rel(M, refs[m]))
    cp.close()


@pytest.mark.parametrize("prec,chunk,steps", [("bf16x3", 1, 0), ("bf16x3", 0, 2), ("tf32x3", 0, 1),
                                               ("tf32x3", 0, 3), ("tf32x3", 2, -1)])
@pytest.mark.parametrize("shape", [SHAPES[0], SHAPES[3], (6, 70, 300, 260)])
def test_restarted_accumulation_mttkrp(prec, chunk, steps, shape):
    """Accumulator restarted every `chunk` K blocks, or every `steps` MMA K steps
    (a K block split unevenly for steps = 3; K tails at every size here)."""
    o, v, X, R = shape
    inp = inputs.make_inputs(o, v, X, R, seed=2)
    refs, abss = _mttkrp_refs(inp.Bvv, inp.tau, inp.factors)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec, acc_chunk=chunk, acc_steps=steps)
    for m in orc.MODES:
        M = cp.mttkrp(m).cpu().numpy()
        check_mttkrp(M, refs[m], abss[m], prec, f"{prec} chunk {chunk} steps {steps} {shape} mode {m}")
        assert _rel(M, refs[m]) < TOL_MTTKRP[prec]
    cp.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_fp64_sweeps_match_oracle(shape):
    o, v, X, R = shape
    inp = inputs.make_inputs(o, v, X, R, seed=2)
    n2, _ = orc.exact_contract(inp.B, inp.tau, o)
    U_ref, lam_ref, hist = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 4, n2)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="fp64", want_eta=True)
    cp.set_normR2(n2)
    fits = cp.sweep(4)
    f = _factors(cp)
    _check_factors(f, U_ref, lam_ref, 1e-8, f"fp64 {shape} after 4 sweeps")
    for k in range(4):
        assert abs(fits[k] - hist[k]["fit"]) < 1e-9
    st = cp.stats()
    assert abs(st["last_eta"] - hist[-1]["eta"]) < 1e-8 * max(hist[-1]["eta"], 1e-3)
    assert st["clamped_pivots"] == sum(h["nclamped"] for h in hist)
    cp.close()


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_exact_contraction_and_energies(shape):
    o, v, X, R = shape
    inp = inputs.make_inputs(o, v, X, R, seed=3)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="fp64")
    n2, E, Rt = cp.exact_contract(want_R=True)
    R_ref = orc.ppl_tensor(inp.Bvv, inp.tau)
    R_abs = orc.ppl_tensor(np.abs(inp.Bvv), np.abs(inp.tau))
    Rg = Rt.cpu().numpy()
    check_abs_bound(Rg, R_ref, R_abs, 1e-12, f"fp64 R {shape}")
    check_columns(Rg.reshape(v * v, o * o), R_ref.reshape(v * v, o * o), 1e-12, f"fp64 R {shape} per (i,j)")
    assert abs(n2 - float(np.sum(R_ref ** 2))) < 1e-12 * n2
    assert abs(E - orc.energy_of_tensor(R_ref, inp.B, o)) < 1e-12 * abs(E)
    lam1 = np.ones(R)
    E_cp = cp.energy()
    assert abs(E_cp - orc.energy_cp(inp.B, o, inp.factors, lam1)) < 1e-12 * abs(E_cp)
    cp.close()


@pytest.mark.parametrize("prec,kcal_tol,ftol", [("bf16x3", 0.1, 2e-2), ("tf32", 0.5, 1e-1), ("tf32x3", 0.01, 2e-4)])
def test_mixed_sweeps_track_fp64_energy(prec, kcal_tol, ftol):
    """Config 0: 20 sweeps in mixed precision from the same start as the FP64
    oracle.  BF16X3 keeps the CP energy within 0.1 kcal/mol of the oracle's;
    TF32 does not (0.12 kcal/mol measured on GB300), so it is held to the
    looser 0.5 and reported as missing the 0.1 kcal/mol bar.  Every factor is
    compared with the oracle's column by column: the per-sweep MTTKRP error
    (about 4e-7, 1e-5 and 6e-4 for TF32X3, BF16X3 and TF32) is amplified by the
    normal-equation solves over 20 sweeps, so ftol is a few hundred times it."""
    inp = inputs.make_inputs(5, 24, 72, 48, seed=0)
    n2, _ = orc.exact_contract(inp.B, inp.tau, 5)
    U_ref, lam_ref, hist = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 20, n2)
    E_ref = orc.energy_cp(inp.B, 5, U_ref, lam_ref)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec)
    cp.set_normR2(n2)
    fits = cp.sweep(20)
    E = cp.energy()
    kcal = 627.509474
    assert abs(E - E_ref) * kcal < kcal_tol
    assert abs(fits[-1] - hist[-1]["fit"]) < 1e-3
    _check_factors(_factors(cp), U_ref, lam_ref, ftol, f"{prec} config 0 after 20 sweeps")
    cp.close()


@pytest.mark.parametrize("prec,ftol", [("tf32x3", 2e-4), ("bf16x3", 2e-2)])
@pytest.mark.parametrize("acc_steps_p", [0, 1])
@pytest.mark.parametrize("dressed", [False, True])
def test_sweeps_over_several_r_chunks(prec, ftol, acc_steps_p, dressed):
    """Config 0 in r-chunks of 16 rank columns (three passes of every chain
    and of the S-build), 10 sweeps against oracle ALS from the same start.
    With acc_steps_p = 0 the S-build reads W_a = B U_a from the mode-b chain of
    the same sweep, transposed per r-chunk into a buffer over all R columns;
    with acc_steps_p = 1 (a different accumulator restart from the chain's) it
    forms W_a itself.  Dressed: D-bar on the b side of every contraction
    (Eq. fulldfB), so the S-build's W_b has another operand than W_a."""
    inp = inputs.make_inputs(5, 24, 72, 48, seed=0)
    Bbar = orc.dress(inp.B, inp.t1, 5) if dressed else None
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 10, 1.0, Bbar=Bbar)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec, r_chunk=16,
                       acc_steps_p=acc_steps_p, dressed=dressed)
    if dressed:
        cp.set_t1(_dev(inp.t1))
    cp.sweep(10)
    _check_factors(_factors(cp), U_ref, lam_ref, ftol,
                   f"{prec} r-chunks of 16, acc_steps_p={acc_steps_p}, dressed={dressed}")
    cp.close()


@pytest.mark.parametrize("kind", ["normal", "uniform"])
def test_seeded_initial_guess_on_the_device(kind):
    """init = NORMAL / UNIFORM draws U_a, U_b, U_i, U_j on the device from the
    counter-based generator of the synthetic inputs (stream 4): NORMAL gives the
    seeded initial factors of inputs.make_factors, UNIFORM the uniforms of the
    same stream (bit-exact: integer mixing and one exact scaling; the normals
    within the last bits of log1p and cos).  Sweeps then match oracle ALS from
    that guess."""
    o, v, X, R, seed = 5, 24, 72, 48, 11
    inp = inputs.make_inputs(o, v, X, R, seed=0)
    n = 2 * v * R + 2 * o * R
    if kind == "normal":
        ref = inputs.make_factors(seed, o, v, R)
    else:
        u = inputs.uniform(seed, inputs.STREAM_FACTORS, n)
        ref, pos = {}, 0
        for m, dim in (("a", v), ("b", v), ("i", o), ("j", o)):
            ref[m] = u[pos:pos + dim * R].reshape(dim, R)
            pos += dim * R
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), R, precision="fp64", init=kind, init_seed=seed)
    f = _factors(cp)
    for m in "abij":
        if kind == "uniform":
            assert np.array_equal(f[m], ref[m]), m
        else:
            assert np.max(np.abs(f[m] - ref[m])) <= 1e-13 * max(1.0, np.max(np.abs(ref[m]))), m
    assert np.all(f["lam"] == 1.0)
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, ref, 3)
    cp.sweep(3)
    _check_factors(_factors(cp), U_ref, lam_ref, 1e-8, f"fp64 sweeps from the {kind} device guess")
    cp.close()


def test_graph_replay_equals_direct_launches():
    inp = inputs.make_inputs(4, 20, 30, 40, seed=5)
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 3)
    out = []
    for use_graph in (False, True):
        cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="bf16x3", use_graph=use_graph)
        cp.sweep(3)
        out.append(_factors(cp))
        cp.close()
    for k in out[0]:
        check_columns(out[1][k].reshape(-1, out[1][k].shape[-1]), out[0][k].reshape(-1, out[0][k].shape[-1]), 1e-6,
                      f"graph vs direct {k}")
    _check_factors(out[1], U_ref, lam_ref, 2e-2, "bf16x3 graph replay vs oracle")


def test_warm_start_set_tau():
    inp = inputs.make_inputs(4, 16, 24, 20, seed=6)
    tau1 = inp.tau + inputs.tau_increment(inp.tau, 1, seed=6)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="fp64")
    cp.sweep(3)
    U0 = {k: t.cpu().numpy().copy() for k, t in cp.factors().items()}
    t1 = _dev(tau1)
    cp.set_tau(t1)
    cp.sweep(2)
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, tau1, {m: U0[m] for m in orc.MODES}, 2, lam0=U0["lam"])
    _check_factors(_factors(cp), U_ref, lam_ref, 1e-9, "warm start after set_tau")
    cp.close()


def test_errors_are_reported_not_raised_in_c():
    inp = inputs.make_inputs(2, 8, 10, 6, seed=7)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="fp64")
    with pytest.raises(binding.PplError) as e:
        cp.fit()
    assert e.value.code == binding.PPL_ENOTREADY
    with pytest.raises(binding.PplError) as e:
        binding.ppl_cpd_mttkrp(cp.h, 7, 0)
    assert e.value.code == binding.PPL_EINVAL
    cp.close()


def test_factors_changed_restarts_from_new_guess():
    inp = inputs.make_inputs(3, 12, 20, 10, seed=8)
    other = inputs.make_factors(99, 3, 12, 10)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="fp64")
    cp.sweep(2)
    cp.set_factors(other)
    cp.sweep(2)
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, other, 2)
    _check_factors(_factors(cp), U_ref, lam_ref, 1e-9, "after factors_changed")
    cp.close()


@pytest.mark.parametrize("rule,eps", [("eta", 0.05), ("dfit", 1e-3)])
def test_solve_sequence_near_optimal_matches_oracle(rule, eps):
    """A CC-like sequence tau_k (k = 0..3), one CPD per tau with a stopping rule,
    Near-Optimal guesses between CPDs: sweep counts and final factors equal the oracle's."""
    inp = inputs.make_inputs(4, 14, 20, 24, seed=9)
    taus = [inp.tau]
    for k in range(1, 4):
        taus.append(taus[-1] + inputs.tau_increment(inp.tau, k, seed=9))
    pol = orc.NearOptimalGuess(inp.factors)
    cp = binding.CpAls(_dev(inp.B), _dev(taus[0]), inp.factors, precision="fp64", want_eta=True)
    cp.set_guess_policy("near_optimal")
    tau_dev = [_dev(t) for t in taus]
    for k, t in enumerate(taus):
        if k:
            cp.set_tau(tau_dev[k])
        n2 = float(np.sum(orc.ppl_tensor(inp.Bvv, t) ** 2))
        cp.set_normR2(n2)
        U0 = pol.start()
        U_ref, lam_ref, hist, its = orc.cp_solve(inp.Bvv, t, U0, 40, rule, eps, n2)
        pol.finish(its)
        n, fits, etas = cp.solve(40, rule, eps)
        assert n == len(hist), (k, n, len(hist))
        _check_factors(_factors(cp), U_ref, lam_ref, 1e-8, f"{rule} solve {k}")
    cp.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_reconstruct_and_symmetrise(prec):
    inp = inputs.make_inputs(3, 13, 17, 70, seed=12)     # R spans two reconstruction chunks
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec)
    cp.sweep(2)
    f = {k: t.cpu().numpy() for k, t in cp.factors().items()}
    R_ref = orc.reconstruct(f, f["lam"])
    R_abs = orc.reconstruct(abs_factors(f), np.abs(f["lam"]))
    check_abs_bound(cp.reconstruct(False).cpu().numpy(), R_ref, R_abs, 1e-13, f"{prec} reconstruction")
    S = cp.reconstruct(True).cpu().numpy()
    check_abs_bound(S, orc.symmetrise(R_ref), orc.symmetrise(R_abs), 1e-13, f"{prec} symmetrised reconstruction")
    assert np.array_equal(S, S.transpose(1, 0, 3, 2)) or _rel(S, S.transpose(1, 0, 3, 2)) < 1e-15
    cp.close()


def test_batch_of_uneven_instances_equals_individual_sweeps():
    shapes = [(4, 40, 120, 96), (6, 56, 168, 130), (5, 24, 72, 48), (8, 64, 192, 200)]
    probs, solo = [], []
    inps = [inputs.make_inputs(*sh, seed=20 + k) for k, sh in enumerate(shapes)]
    for inp in inps:
        probs.append(binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="bf16x3"))
        solo.append(binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="bf16x3"))
    batch = binding.Batch(probs, nstreams=3)
    batch.sweep(3)
    for p, q in zip(probs, solo):
        q.sweep(3)
        fp, fq = _factors(p), _factors(q)
        for k in fp:
            check_columns(fp[k].reshape(-1, fp[k].shape[-1]), fq[k].reshape(-1, fq[k].shape[-1]), 1e-12,
                          f"batch vs solo {k}")
    # the batch graph solves each mode of all instances in one launch (plus its
    # barrier reset) and runs contractions of equal depth in grouped launches: at
    # least the first contraction of every instance (T of mode a) shares one
    n = len(probs)
    solo_kernels = sum(int(q.stats()["kernels_per_sweep"]) for q in solo)
    assert batch.kernels_per_sweep() <= solo_kernels - 4 * n + 8 - (n - 1), (batch.kernels_per_sweep(), solo_kernels)
    batch.close()
    for p in probs + solo:
        p.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("tf32x3", 2e-4)])
def test_batch_of_uneven_instances_against_oracle(prec, tol):
    """Four uneven instances swept together from one graph (each on its share of
    the SMs): after three sweeps every instance's factors equal the oracle's ALS
    from the same start, column by column (the tolerance of the FP64 form, or
    the mixed-precision factor tolerance of the sweep tests)."""
    shapes = [(4, 40, 120, 96), (6, 56, 168, 130), (5, 24, 72, 48), (8, 64, 192, 200)]
    inps = [inputs.make_inputs(*sh, seed=20 + k) for k, sh in enumerate(shapes)]
    probs = [binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec) for inp in inps]
    batch = binding.Batch(probs, nstreams=3)
    batch.sweep(3)
    for k, (inp, p) in enumerate(zip(inps, probs)):
        U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 3)
        _check_factors(_factors(p), U_ref, lam_ref, tol, f"{prec} batch instance {k} {shapes[k]}")
    batch.close()
    for p in probs:
        p.close()


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_autotune_picks_a_chunk_and_keeps_results(prec):
    """The autotuned r-chunk (several passes of the chain, a ragged last one)
    gives MTTKRPs equal to the oracle's element by element, and the same sweeps
    as the planned chunk."""
    inp = inputs.make_inputs(6, 48, 144, 300, seed=30)
    refs, abss = _mttkrp_refs(inp.Bvv, inp.tau, inp.factors)
    a = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec)
    rc = a.autotune()
    assert 16 <= rc <= 1024 and (rc % 16 == 0 or rc == 300)   # a multiple of 16, or all of R
    for m in orc.MODES:
        check_mttkrp(a.mttkrp(m).cpu().numpy(), refs[m], abss[m], prec, f"{prec} autotuned r-chunk {rc} mode {m}")
    b = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec, r_chunk=48)
    for m in orc.MODES:
        check_mttkrp(b.mttkrp(m).cpu().numpy(), refs[m], abss[m], prec, f"{prec} r-chunk 48 mode {m}")
    a.sweep(2)
    b.sweep(2)
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 2)
    _check_factors(_factors(a), U_ref, lam_ref, 2e-2 if prec == "bf16x3" else 2e-4, f"{prec} autotuned sweeps")
    _check_factors(_factors(b), U_ref, lam_ref, 2e-2 if prec == "bf16x3" else 2e-4, f"{prec} r-chunk 48 sweeps")
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "tf32x3"])
def test_dressed_mttkrp_sweeps_and_exact(prec):
    inp = inputs.make_inputs(4, 21, 30, 40, seed=41)
    Bbar = orc.dress(inp.B, inp.t1, inp.o)
    refs, abss = _mttkrp_refs(inp.Bvv, inp.tau, inp.factors, Bbar)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec, dressed=True)
    cp.set_t1(_dev(inp.t1))
    for m in orc.MODES:
        check_mttkrp(cp.mttkrp(m).cpu().numpy(), refs[m], abss[m], prec, f"{prec} dressed mode {m}")
    n2, E, Rt = cp.exact_contract(want_R=True)
    R_ref = orc.ppl_tensor(inp.Bvv, inp.tau, Bbar)
    R_abs = orc.ppl_tensor(np.abs(inp.Bvv), np.abs(inp.tau), np.abs(Bbar))
    check_abs_bound(Rt.cpu().numpy(), R_ref, R_abs, 1e-12, "dressed R (FP64)")
    assert abs(E - orc.energy_of_tensor(R_ref, inp.B, inp.o)) < 1e-12 * abs(E)
    U_ref, lam_ref, hist = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 3, n2, Bbar=Bbar)
    fits = cp.sweep(3)
    ftol = {"fp64": 1e-8, "tf32x3": 2e-4, "bf16x3": 2e-2}[prec]
    _check_factors(_factors(cp), U_ref, lam_ref, ftol, f"{prec} dressed sweeps")
    assert abs(fits[-1] - hist[-1]["fit"]) < (1e-9 if prec == "fp64" else 1e-4)
    cp.set_t1(None)                       # undressed again: back to the symmetric tensor
    f = _factors(cp)
    r2, a2 = _mttkrp_refs(inp.Bvv, inp.tau, f)
    check_mttkrp(cp.mttkrp("a").cpu().numpy(), r2["a"], a2["a"], prec, f"{prec} undressed again mode a")
    cp.close()


@pytest.mark.parametrize("prec,tol", [("bf16x3", 1e-4), ("tf32", 4e-3), ("tf32x3", 1e-5)])
@pytest.mark.parametrize("dressed", [False, True])
def test_exact_contraction_on_tensor_cores(prec, tol, dressed):
    """R formed on the tensor cores: element by element within the bound of its
    two contractions (G = B.D-bar with K = X, then R = G tau with K = v^2 split
    over K), and within tol of the largest |R| of every (i, j) column."""
    inp = inputs.make_inputs(5, 26, 70, 30, seed=44)
    Bbar = orc.dress(inp.B, inp.t1, inp.o) if dressed else None
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision=prec, dressed=dressed)
    if dressed:
        cp.set_t1(_dev(inp.t1))
    n2, E, Rt = cp.exact_contract(want_R=True, mixed=True)
    R_ref = orc.ppl_tensor(inp.Bvv, inp.tau, Bbar)
    R_abs = orc.ppl_tensor(np.abs(inp.Bvv), np.abs(inp.tau), None if Bbar is None else np.abs(Bbar))
    Rg = Rt.cpu().numpy()
    o, v = inp.o, inp.Bvv.shape[1]
    check_abs_bound(Rg, R_ref, R_abs, GAMMA[prec], f"{prec} R on tensor cores")
    check_columns(Rg.reshape(v * v, o * o), R_ref.reshape(v * v, o * o), COLTOL[prec], f"{prec} R per (i,j)")
    assert _rel(Rg, R_ref) < tol
    assert abs(n2 - float(np.sum(R_ref ** 2))) < 2 * tol * n2
    E_ref = orc.energy_of_tensor(R_ref, inp.B, inp.o)
    assert abs(E - E_ref) < 2 * tol * abs(E_ref)
    cp.close()


def test_full_size_benchmark_instance():
    """o=20 v=200 X=600 R=800, the benchmark's instance, in the configuration bench.py
    times (graph replay, r-chunk from the autotuner): every MTTKRP against the oracle,
    element by element; then, after two sweeps, the library's <R, R~> and ||R~||^2
    against the oracle's values of the same quantities evaluated from the library's
    own factors."""
    inp = inputs.make_inputs(20, 200, 600, 800, seed=0)
    refs, abss = _mttkrp_refs(inp.Bvv, inp.tau, inp.factors)
    B, tau = _dev(inp.B), _dev(inp.tau)
    for prec in ("tf32x3", "bf16x3"):
        cp = binding.CpAls(B, tau, inp.factors, precision=prec)
        cp.autotune()
        for m in orc.MODES:
            M = cp.mttkrp(m).cpu().numpy()
            check_mttkrp(M, refs[m], abss[m], prec, f"{prec} o=20 v=200 X=600 R=800 mode {m}")
            assert _rel(M, refs[m]) < TOL_MTTKRP[prec], (prec, m)
        cp.sweep(2, want_hist=False)
        st = cp.stats()
        f = _factors(cp)
        M_j = orc.mttkrp(inp.Bvv, inp.tau, f, "j")
        inner = orc.inner_from_mttkrp(M_j, f["j"], f["lam"])
        norm2 = orc.cp_norm2(f, f["lam"])
        assert abs(st["last_inner"] - inner) < 4 * TOL_MTTKRP[prec] * abs(inner), (prec, st["last_inner"], inner)
        assert abs(st["last_norm2"] - norm2) < 1e-10 * norm2, (prec, st["last_norm2"], norm2)
        cp.close()


@pytest.mark.parametrize("shape", [(40, 400, 1200, 1600), (60, 600, 1800, 2400)])
def test_full_size_sampled_columns(shape):
    """The larger configured sizes (o, v, X, R) = (40, 400, 1200, 1600) and
    (60, 600, 1800, 2400), TF32X3 with the autotuned r-chunk as bench.py runs them:
    every mode's MTTKRP on the first and last rank column of every r-chunk
    (including the ragged last chunk) against the oracle evaluated on those columns
    alone (column r of an MTTKRP depends only on column r of the factors), element
    by element."""
    o, v, X, R = shape
    B, tau, fac = inputs.make_inputs_torch(o, v, X, R, seed=5, device="cuda")
    cp = binding.CpAls(B, tau, fac, precision="tf32x3")
    rc = cp.autotune()
    M = {m: cp.mttkrp(m).cpu().numpy() for m in orc.MODES}
    cp.close()
    edges = sorted({c for r0 in range(0, R, rc) for c in (r0, min(R, r0 + rc) - 1)})
    cols = np.array(edges[:8] + edges[-4:] if len(edges) > 12 else edges)
    cols = np.unique(cols)
    Bh = B.cpu().numpy()
    del B
    tau_h = tau.cpu().numpy()
    del tau
    torch.cuda.empty_cache()
    Bvv = np.ascontiguousarray(Bh[:, o:, o:])
    sub = {m: np.ascontiguousarray(fac[m][:, cols]) for m in orc.MODES}
    refs, abss = _mttkrp_refs(Bvv, tau_h, sub)
    for m in orc.MODES:
        got = M[m][:, cols]
        check_mttkrp(got, refs[m], abss[m], "tf32x3", f"{shape} r-chunk {rc} columns {list(cols)} mode {m}")
        assert _rel(got, refs[m]) < TOL_MTTKRP["tf32x3"], (shape, m, _rel(got, refs[m]))


@pytest.mark.parametrize("use_graph", [False, True])
def test_bounded_wait_expires_and_handle_recovers(use_graph):
    """A bounded device wait that runs out.  One block of the cooperative solve
    is told (through a flag armed from the host) to withhold its first grid
    barrier arrival; the other blocks' wait, limited to 20 ms here, runs out,
    they raise the abort flag, every block returns, and the sweep reports
    PPL_ETIMEOUT, counted in stats.timeouts.  No kernel is left waiting: the
    withholding block itself waits for the abort with a bound.  The same handle,
    reset to the initial guess, then sweeps normally and matches the oracle."""
    import time
    inp = inputs.make_inputs(5, 24, 72, 48, seed=0)
    cp = binding.CpAls(_dev(inp.B), _dev(inp.tau), inp.factors, precision="tf32x3", use_graph=use_graph,
                       wait_limit_us=20000)
    if use_graph:
        cp.sweep(1)                      # capture the sweep graph first; the flag is read at run time
        cp.set_factors(inp.factors)
    assert cp.stats()["timeouts"] == 0
    binding.ppl_cpd_inject_wait_timeout(cp.h)
    t0 = time.perf_counter()
    with pytest.raises(binding.PplError) as e:
        cp.sweep(1)
    elapsed = time.perf_counter() - t0
    assert e.value.code == binding.PPL_ETIMEOUT, str(e.value)
    assert elapsed < 5.0, elapsed
    assert cp.stats()["timeouts"] == 1
    cp.set_factors(inp.factors)
    cp.sweep(2)
    assert cp.stats()["timeouts"] == 1
    U_ref, lam_ref, _ = orc.cp_als(inp.Bvv, inp.tau, inp.factors, 2)
    _check_factors(_factors(cp), U_ref, lam_ref, 2e-4, f"tf32x3 sweeps after a timeout (graph {use_graph})")
    cp.close()


def test_pivot_reciprocal_within_two_ulp():
    """The Cholesky inverts its pivots with the PTX approximate FP64 reciprocal
    refined by two Newton-Raphson steps (each squares the relative error).  Over
    a log-spaced sweep of positive normal doubles from 1e-300 to 1e300, values
    just above and below powers of two, random mantissas, and pivots of the size
    of the clamp tolerance (2^-52 R max V_kk for R up to 2400), the result is
    within two ulps of the correctly rounded 1/d."""
    rng = np.random.default_rng(3)
    d = [np.logspace(-300, 300, 120001)]
    e = np.arange(-990, 991, 7, dtype=np.float64)
    d.append(np.ldexp(1.0, e.astype(int)))
    d.append(np.nextafter(np.ldexp(1.0, e.astype(int)), 0.0))
    d.append(np.nextafter(np.ldexp(1.0, e.astype(int)), np.inf))
    d.append(rng.uniform(1.0, 2.0, 20000) * np.ldexp(1.0, rng.integers(-900, 900, 20000)))
    d.append(2.0 ** -52 * np.array([1, 48, 800, 1600, 2400], dtype=np.float64)[:, None]
             * np.logspace(-6, 6, 101)[None, :])
    d = np.concatenate([x.ravel() for x in d])
    d = d[(d > 1e-300) & (d < 1e300)]
    dev = torch.from_numpy(d).cuda()
    out = torch.empty_like(dev)
    rc = binding.lib().ppl_test_reciprocal(dev.data_ptr(), out.data_ptr(), dev.numel(),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == binding.PPL_OK
    got = out.cpu().numpy()
    ref = 1.0 / d
    ulps = np.abs(got - ref) / np.spacing(ref)
    w = int(np.argmax(ulps))
    assert ulps[w] <= 2.0, (d[w], got[w], ref[w], ulps[w])
