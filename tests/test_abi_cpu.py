"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/ppl_cpd.h declares, and rejects bad arguments
before touching the device."""

import ctypes
import os
import re

import pytest

from paper_2503_10380_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    try:
        __graft_entry__.build()
    except RuntimeError as e:   # no nvcc on this machine
        pytest.skip(str(e))
    return binding.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ppl_\w+)\s*\(", txt, flags=re.M))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_workspace_size_validates(lib):
    o = binding.make_opts("bf16x3")
    with pytest.raises(binding.PplError) as e:
        binding.ppl_cpd_workspace_size(0, 24, 72, 48, o)
    assert e.value.code == binding.PPL_EINVAL
    o.precision = 9
    with pytest.raises(binding.PplError):
        binding.ppl_cpd_workspace_size(5, 24, 72, 48, o)


def test_workspace_grows_with_rank_and_precision_layout(lib):
    f64 = binding.ppl_cpd_workspace_size(5, 24, 72, 48, binding.make_opts("fp64"))
    b16 = binding.ppl_cpd_workspace_size(5, 24, 72, 48, binding.make_opts("bf16x3"))
    t32 = binding.ppl_cpd_workspace_size(5, 24, 72, 48, binding.make_opts("tf32"))
    big = binding.ppl_cpd_workspace_size(5, 24, 72, 96, binding.make_opts("bf16x3"))
    # both 4-byte operand elements; bf16 K panels are 64 elements wide against 32, so
    # the bf16 layout pads at least as much
    assert b16 >= t32 and big > b16 and f64 > 0


def test_workspace_follows_the_planner_options(lib):
    ws = binding.ppl_cpd_workspace_size
    shape = (20, 200, 600, 800)
    b16 = ws(*shape, binding.make_opts("bf16x3"))
    t3 = ws(*shape, binding.make_opts("tf32x3"))
    assert t3 > b16                                   # 8-byte operand elements against 4
    # explicit r-chunks: more rank columns per pass need wider chunk buffers, capped at 1024
    sizes = [ws(*shape, binding.make_opts("tf32x3", r_chunk=rc)) for rc in (64, 256, 800)]
    assert sizes[0] < sizes[1] < sizes[2]
    big = (20, 200, 600, 3000)
    assert ws(*big, binding.make_opts("tf32x3", r_chunk=1024)) == ws(*big, binding.make_opts("tf32x3", r_chunk=4096))
    # automatic chunk: all of R while one [rc][X][v] operand buffer stays within 8 GiB ...
    assert t3 == ws(*shape, binding.make_opts("tf32x3", r_chunk=800))
    # ... and equal chunks under that budget otherwise (X v 8 bytes = 8.64 MB per column: 3 x 800)
    cfg4 = (60, 600, 1800, 2400)
    assert ws(*cfg4, binding.make_opts("tf32x3")) == ws(*cfg4, binding.make_opts("tf32x3", r_chunk=800))
    # the dressed D-bar takes room; accumulator restarts take none
    assert ws(*shape, binding.make_opts("tf32x3", dressed=True)) > t3
    assert ws(*shape, binding.make_opts("tf32x3", acc_chunk=2, acc_steps=1)) == t3


def test_init_rejects_small_workspace_and_null(lib):
    opts = binding.make_opts("fp64")
    need = binding.ppl_cpd_workspace_size(5, 24, 72, 48, opts)
    h = ctypes.c_void_p()
    fake = 1 << 20   # never dereferenced: the checks run before any CUDA call
    rc = lib.ppl_cpd_init(ctypes.byref(h), 5, 24, 72, 48, fake, fake, fake, fake, need - 1,
                          ctypes.byref(opts), None)
    assert rc == binding.PPL_ENOMEM
    assert b"needs" in lib.ppl_last_error(None)
    rc = lib.ppl_cpd_init(ctypes.byref(h), 5, 24, 72, 48, None, fake, fake, fake, need, ctypes.byref(opts), None)
    assert rc == binding.PPL_EINVAL
    rc = lib.ppl_cpd_init(ctypes.byref(h), 5, 24, 72, 48, fake, fake, fake, fake + 8, need, ctypes.byref(opts), None)
    assert rc == binding.PPL_EINVAL   # misaligned workspace
    assert lib.ppl_cpd_destroy(None) == binding.PPL_OK


def test_init_guess_options(lib):
    """The options struct keeps its size (16 ints: init and init_seed took two
    of the reserved words) and an unknown guess kind is refused before any CUDA
    call."""
    assert ctypes.sizeof(binding.ppl_cpd_opts) == 16 * 4
    assert binding.ppl_cpd_opts.init.offset == 10 * 4 and binding.ppl_cpd_opts.init_seed.offset == 11 * 4
    opts = binding.make_opts("fp64", init="normal", init_seed=-1)
    assert opts.init == 1 and opts.init_seed == -1          # the seed is taken as unsigned by the library
    opts.init = 7
    need = binding.ppl_cpd_workspace_size(5, 24, 72, 48, opts)
    h = ctypes.c_void_p()
    fake = 1 << 20
    rc = lib.ppl_cpd_init(ctypes.byref(h), 5, 24, 72, 48, fake, fake, fake, fake, need, ctypes.byref(opts), None)
    assert rc == binding.PPL_EINVAL
    assert b"initial guess" in lib.ppl_last_error(None)


def test_handle_calls_reject_null_handle(lib):
    x = ctypes.c_double()
    assert lib.ppl_cpd_fit(None, ctypes.byref(x)) == binding.PPL_EINVAL
    assert lib.ppl_cpd_sweep(None, 1, None) == binding.PPL_EINVAL
    assert lib.ppl_cpd_mttkrp(None, 0, None) == binding.PPL_EINVAL
