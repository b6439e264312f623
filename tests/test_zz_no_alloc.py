"""ptx_llk_static: the log-likelihood entry point that allocates nothing.

Callers that cannot allocate device memory (code inside a host application
that owns all device memory, or a loop that must not enter an allocator) get
the exact Poisson LLK from ptx_llk_static, whose working memory is a fixed
file-scope device array.  It must agree with the handle-based ptx_llk (same
kernels, so to within the 1e-5 relative tolerance of the other GPU tests and in
practice exactly), including on a second call in a row that reuses the array,
and with the FP64 oracle's LLK.  A masked call followed by an unmasked one must
not see the first call's mask (the array keeps the last call's contents).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synthetic import make_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL1 = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2008_11511_gb300 import build as b
    b.build()
    from paper_2008_11511_gb300 import _lib
    return _lib.load()


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def _static_llk(lib, s, obj, probe, iobs, out):
    pos = np.ascontiguousarray(s.positions.astype(np.int32))
    mask = np.ascontiguousarray(s.mask.astype(np.uint8)) if s.mask.any() else None
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.ptx_llk_static(s.N, s.K, s.J, s.Ho, s.Wo, ctypes.c_void_p(obj.data_ptr()),
                            ctypes.c_void_p(probe.data_ptr()), ctypes.c_void_p(pos.ctypes.data),
                            ctypes.c_void_p(iobs.data_ptr()),
                            ctypes.c_void_p(mask.ctypes.data) if mask is not None else None,
                            ctypes.c_void_p(out.data_ptr()), stream)
    return st


@pytest.mark.parametrize("cfg,J,over", [("ap64", 100, {}), ("dm256", 300, {"Ho": 768, "Wo": 768}),
                                         ("modes512", 12, {"Ho": 900, "Wo": 900})])
def test_static_llk_matches_handle_llk_twice(lib, cfg, J, over):
    from paper_2008_11511_gb300 import Ptycho
    s = make_config(cfg, J=J, **over)
    obj, probe, iobs = _dev(s.obj0), _dev(s.probe0), _dev(s.iobs)
    pb = Ptycho(obj, probe, iobs, s.positions, s.mask, with_psi=False)
    ref = float(pb.llk())
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for i in range(2):
        st = _static_llk(lib, s, obj, probe, iobs, out[i:i + 1])
        assert st == 0, lib.ptx_last_error()
    got = out.cpu().numpy()
    assert abs(got[0] - ref) <= TOL1 * abs(ref), (got, ref)
    assert abs(got[1] - ref) <= TOL1 * abs(ref), (got, ref)
    pb.close()


def test_static_llk_rejects_sizes_beyond_its_array(lib):
    s = make_config("ap64", J=10)
    obj, probe, iobs = _dev(s.obj0), _dev(s.probe0), _dev(s.iobs)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = make_config("ap64", J=10)
    big.J = 70000
    big.positions = np.zeros((70000, 2), np.int32)
    assert _static_llk(lib, big, obj, probe, iobs, out) == 2  # PTX_ERR_UNSUPPORTED
    assert b"static scratch" in lib.ptx_last_error()
    wide = make_config("ap64", J=10)
    wide.N, wide.K = 512, 8
    wide.Ho = wide.Wo = 512
    wide.positions = np.zeros((10, 2), np.int32)
    assert _static_llk(lib, wide, obj, probe, iobs, out) == 2
    assert b"static scratch" in lib.ptx_last_error()
    assert _static_llk(lib, s, obj, probe, iobs, out) == 0


def _warm(cfg, J, **over):
    """The oracle's state after one AP cycle from the configured start (where the
    single-precision far field resolves the whole detector), as complex64."""
    s = make_config(cfg, J=J, **over)
    o, p, _ = oracle.ap_cycle(s.obj0, s.probe0, oracle.Data.make(s.iobs, s.positions, s.mask))
    return s, o.astype(np.complex64), p.astype(np.complex64)


def test_static_llk_matches_the_oracle(lib):
    s, o, p = _warm("ap64", 100, mask_fraction=0.03)
    assert s.mask.any()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    obj, probe, iobs = _dev(o), _dev(p), _dev(s.iobs)
    for i in range(2):
        assert _static_llk(lib, s, obj, probe, iobs, out[i:i + 1]) == 0, lib.ptx_last_error()
    ref = oracle.llk(o, p, oracle.Data.make(s.iobs, s.positions, s.mask))
    got = out.cpu().numpy()
    assert abs(got[0] - ref) <= TOL1 * abs(ref) and abs(got[1] - ref) <= TOL1 * abs(ref), (got, ref)


def test_static_llk_masked_then_unmasked_call(lib):
    """The second, unmasked call in the same stream must see no mask: the masked
    call clears its mask region of the shared array behind it."""
    from paper_2008_11511_gb300 import Ptycho
    s, o, p = _warm("ap64", 60, mask_fraction=0.05)
    assert s.mask.any()
    obj, probe, iobs = _dev(o), _dev(p), _dev(s.iobs)
    nomask = make_config("ap64", J=60, mask_fraction=0.05)
    nomask.mask = np.zeros_like(s.mask)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert _static_llk(lib, s, obj, probe, iobs, out[0:1]) == 0, lib.ptx_last_error()
    assert _static_llk(lib, nomask, obj, probe, iobs, out[1:2]) == 0, lib.ptx_last_error()
    got = out.cpu().numpy()
    pb_m = Ptycho(obj, probe, iobs, s.positions, s.mask, with_psi=False)
    pb_u = Ptycho(obj, probe, iobs, s.positions, None, with_psi=False)
    ref_m, ref_u = float(pb_m.llk()), float(pb_u.llk())
    pb_m.close()
    pb_u.close()
    assert abs(ref_u - ref_m) > 1e-3 * abs(ref_u)  # the mask matters on this case
    assert abs(got[0] - ref_m) <= TOL1 * abs(ref_m), (got, ref_m)
    assert abs(got[1] - ref_u) <= TOL1 * abs(ref_u), (got, ref_u)
    ref_o = oracle.llk(o, p, oracle.Data.make(s.iobs, s.positions, None))
    assert abs(got[1] - ref_o) <= TOL1 * abs(ref_o), (got, ref_o)
