"""The allocation-free CP energy, ppl_cp_energy_static.

Some callers cannot allocate device memory when they need the energy: a
framework that owns all device memory through its own pooling allocator and
cannot hand a workspace through, or latency-bound code that must not call
cudaMalloc / cudaFree mid-solve because they can synchronise the device.
This entry point keeps its scratch in a fixed array inside the library.  The
test calls it through the C ABI twice in a row (the array keeps the previous
call's contents, so the second call checks that nothing leaks between calls)
and compares with ppl_cpd_energy, the workspace-based entry point, to the
FP64 tolerance the other energy tests use.  It lives in its own file so that
pytest collects it last.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_10380_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("shape", [(5, 24, 72, 48), (20, 24, 72, 800)])
def test_static_energy_matches_workspace_energy_twice(shape):
    o, v, X, R = shape     # the second shape needs three chunks of Q in the static array
    inp = inputs.make_inputs(o, v, X, R, seed=11)
    B = torch.from_numpy(inp.B).cuda()
    tau = torch.from_numpy(inp.tau).cuda()
    cp = binding.CpAls(B, tau, inp.factors, precision="fp64")
    cp.sweep(2)
    E_ref = cp.energy()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        E = binding.ppl_cp_energy_static(o, v, X, R, B.data_ptr(), cp.fac.data_ptr(), stream)
        assert abs(E - E_ref) <= 1e-12 * abs(E_ref)
    cp.close()


def test_static_energy_rejects_sizes_beyond_its_array():
    o, R = 1000, 1000      # 2 * o * R * 8 bytes exceed the array; refused before any device work
    # real device buffers rather than made-up addresses; the call must refuse the
    # sizes before it reads them
    B = torch.zeros(1, dtype=torch.float64, device="cuda")
    fac = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(binding.PplError) as e:
        binding.ppl_cp_energy_static(o, 10, 10, R, B.data_ptr(), fac.data_ptr(), None)
    assert e.value.code == binding.PPL_EINVAL
    assert "static scratch limit" in str(e.value)
