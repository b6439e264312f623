"""ptx_llk_static: the log-likelihood entry point that allocates nothing.

Callers that cannot allocate device memory (code inside a host application
that owns all device memory, or a loop that must not enter an allocator) get
the exact Poisson LLK from ptx_llk_static, whose working memory is a fixed
file-scope device array.  It must agree with the handle-based ptx_llk (same
kernels, so to within the 1e-5 relative tolerance of the other GPU tests and in
practice exactly), including on a second call in a row that reuses the array.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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
