"""The C-ABI library loads, exports every symbol include/ptycho.h declares, and
rejects bad arguments on the host (no device work: these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ptycho.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2008_11511_gb300 import build as b
    b.build()
    from paper_2008_11511_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ptx_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ptx_create", "ptx_ap_cycles", "ptx_dm_cycles", "ptx_llk", "ptx_ml_grad", "ptx_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2008_11511_gb300._lib import EXPORTS
    names = declared_functions()
    assert sorted(EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def _problem(N=64, K=1, J=3, Ho=128, Wo=100, positions=None):
    from paper_2008_11511_gb300._lib import Problem
    pos = np.array(positions if positions is not None else [[0, 0], [10, 20], [Ho - N, Wo - N]],
                   dtype=np.int32)
    p = Problem(N=N, K=K, J=len(pos), Ho=Ho, Wo=Wo, obj=0x1000, probe=0x2000, positions=pos.ctypes.data,
                iobs=0x3000, mask=None, psi=None)
    return p, pos


def _ws(lib, p):
    n = ctypes.c_size_t(0)
    st = lib.ptx_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(n))
    return st, n.value


def test_workspace_bytes_and_argument_checks(lib):
    from paper_2008_11511_gb300._lib import STATUS_NAMES
    p, pos = _problem()
    st, n = _ws(lib, p)
    assert st == 0 and n > 128 * 100 * 16
    # unsupported frame size
    p2, pos2 = _problem(N=100, Ho=200, Wo=200, positions=[[0, 0]])
    st, _ = _ws(lib, p2)
    assert STATUS_NAMES[st] == "PTX_ERR_UNSUPPORTED"
    assert b"not supported" in lib.ptx_last_error()
    # out-of-bounds position (one past the last valid row)
    p3, pos3 = _problem(positions=[[0, 0], [128 - 64 + 1, 0]])
    st, _ = _ws(lib, p3)
    assert STATUS_NAMES[st] == "PTX_ERR_OUT_OF_BOUNDS"
    p4, pos4 = _problem(positions=[[0, -1]])
    st, _ = _ws(lib, p4)
    assert STATUS_NAMES[st] == "PTX_ERR_OUT_OF_BOUNDS"
    # too many modes, zero modes, object smaller than the frame
    p5, pos5 = _problem(K=9)
    assert STATUS_NAMES[_ws(lib, p5)[0]] == "PTX_ERR_UNSUPPORTED"
    p6, pos6 = _problem(K=0)
    assert STATUS_NAMES[_ws(lib, p6)[0]] == "PTX_ERR_INVALID_ARG"
    p7, pos7 = _problem(Ho=32, Wo=32, positions=[[0, 0]])
    assert STATUS_NAMES[_ws(lib, p7)[0]] == "PTX_ERR_INVALID_ARG"
    # null arguments
    n = ctypes.c_size_t()
    assert STATUS_NAMES[lib.ptx_workspace_bytes(None, 1, ctypes.byref(n))] == "PTX_ERR_INVALID_ARG"
    p8, pos8 = _problem()
    p8.iobs = None
    assert STATUS_NAMES[_ws(lib, p8)[0]] == "PTX_ERR_INVALID_ARG"


def test_work_stack_sizing(lib):
    """The Fourier work stack: 64 MB for frames of less than 4 MB of spectra
    (two lanes of 64 frames at 256^2), at least 21 frames per lane for larger
    ones (three-mode 512^2 frames of 6 MB: 252 MB); a scan of fewer frames
    takes only what its frames need."""
    mb = 1 << 20
    f512k3 = 3 * 512 * 512 * 8

    def ws(N, K, Ho, Wo, positions):
        p, pos = _problem(N=N, K=K, Ho=Ho, Wo=Wo, positions=positions)  # pos must outlive the call
        st, n = _ws(lib, p)
        assert st == 0
        return n

    pos256 = [[(7 * i) % 200, (13 * i) % 200] for i in range(200)]
    n256 = ws(256, 1, 456, 456, pos256)
    assert 64 * mb < n256 < 96 * mb
    pos512 = [[(7 * i) % 80, (13 * i) % 80] for i in range(60)]
    n512k3 = ws(512, 3, 592, 592, pos512)
    assert 2 * 21 * f512k3 < n512k3 < 2 * 21 * f512k3 + 64 * mb
    n512k3s = ws(512, 3, 592, 592, pos512[:4])  # four frames: a stack of four frames per lane
    assert 2 * 4 * f512k3 < n512k3s < 2 * 4 * f512k3 + 64 * mb
    n512k1 = ws(512, 1, 592, 592, pos512)  # 2 MB frames keep the 64 MB stack
    assert 64 * mb < n512k1 < 96 * mb


def test_encode_counts8_matches_its_definition(lib):
    """ptx_encode_counts8 (host): out8 = min(c, 255), escapes = every index
    with c >= 255 in increasing order with its count; boundaries 254 / 255 /
    256 / 65535, an empty input, the count-only query and a too-small
    capacity."""
    from paper_2008_11511_gb300._lib import STATUS_NAMES
    from paper_2008_11511_gb300 import encode_counts8
    rng = np.random.default_rng(7)
    c = rng.poisson(3.0, size=(5, 37, 41)).astype(np.uint16)
    c[0, 0, :6] = [0, 254, 255, 256, 65535, 1]
    c[4, -1, -3:] = [255, 65534, 300]
    out8, idx, val = encode_counts8(c)
    flat = c.ravel()
    want_idx = np.nonzero(flat >= 255)[0]
    assert out8.dtype == np.uint8 and out8.shape == c.shape
    np.testing.assert_array_equal(out8, np.minimum(c, 255).astype(np.uint8))
    np.testing.assert_array_equal(idx, want_idx.astype(np.uint32))
    np.testing.assert_array_equal(val, flat[want_idx])
    # decoding on the host by the definition gives the counts back
    dec = out8.ravel().astype(np.uint32)
    dec[idx] = val
    np.testing.assert_array_equal(dec, flat)
    # empty input; count-only query; too small a capacity
    o0, i0, v0 = encode_counts8(np.zeros((0,), dtype=np.uint16))
    assert o0.size == 0 and i0.size == 0 and v0.size == 0
    n_esc = ctypes.c_size_t(0)
    assert lib.ptx_encode_counts8(flat.ctypes.data, flat.size, None, None, None, 0, ctypes.byref(n_esc)) == 0
    assert n_esc.value == want_idx.size
    o = np.empty(flat.size, dtype=np.uint8)
    ib = np.empty(2, dtype=np.uint32)
    vb = np.empty(2, dtype=np.uint16)
    st = lib.ptx_encode_counts8(flat.ctypes.data, flat.size, o.ctypes.data, ib.ctypes.data, vb.ctypes.data, 2,
                                ctypes.byref(n_esc))
    assert STATUS_NAMES[st] == "PTX_ERR_OUT_OF_BOUNDS" and n_esc.value == want_idx.size
    np.testing.assert_array_equal(ib, want_idx[:2].astype(np.uint32))
    assert STATUS_NAMES[lib.ptx_encode_counts8(None, 10, None, None, None, 0, ctypes.byref(n_esc))] == \
        "PTX_ERR_INVALID_ARG"


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2008_11511_gb300._lib import STATUS_NAMES
    assert STATUS_NAMES[lib.ptx_ap_cycles(None, 1, 3, None, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_dm_cycles(None, 1, 3, None, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_llk(None, None, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_ml_grad(None, None, None, None, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_set_param(None, b"alpha_obj", 0.1)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_fft2(None, 1, 64, -1, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_fft2(ctypes.c_void_p(0x1000), 1, 100, -1, None)] == "PTX_ERR_UNSUPPORTED"
    assert STATUS_NAMES[lib.ptx_fft2(ctypes.c_void_p(0x1000), 1, 64, 2, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_wait_selftest(None, 1000, None)] == "PTX_ERR_INVALID_ARG"
    assert STATUS_NAMES[lib.ptx_counts_to_float(None, None, 0, None)] == "PTX_OK"
    assert STATUS_NAMES[lib.ptx_counts_to_float(None, None, 5, None)] == "PTX_ERR_INVALID_ARG"
    lib.ptx_destroy(None)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2008_11511_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the compiled library the binding raises; there is no fallback
    path that computes anything on the host."""
    import paper_2008_11511_gb300._lib as L
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="libptycho.so not found"):
        L.load(str(tmp_path / "libptycho.so"))


def test_python_api_imports_without_a_gpu():
    from paper_2008_11511_gb300 import Ptycho, PtychoError, PtychoLLK, fft2  # noqa: F401
    import paper_2008_11511_gb300.ptycho as m
    assert m.Ptycho is Ptycho


# ---------------------------------------------------------------- position refinement, host step

def test_oracle_refine_positions_step_pins():
    """The oracle's host step of position refinement against hand-worked cases:
    0.3 px per step moves the frame after the second step (10.6 rounds to 11),
    a 5 px shift is clipped to max_shift, the object edge stops the position,
    and exact halves round to even."""
    from oracle import ptycho as orc
    pos = np.array([[10.0, 10.0]])
    pos, ip = orc.refine_positions_step(pos, np.array([[0.3, -0.3]]), 1.0, 2.0, 50, 50)
    assert np.allclose(pos, [[10.3, 9.7]]) and ip.tolist() == [[10, 10]]
    pos, ip = orc.refine_positions_step(pos, np.array([[0.3, -0.3]]), 1.0, 2.0, 50, 50)
    assert np.allclose(pos, [[10.6, 9.4]]) and ip.tolist() == [[11, 9]]
    pos, ip = orc.refine_positions_step(np.array([[20.0, 20.0]]), np.array([[5.0, -5.0]]), 1.0, 2.0, 50, 50)
    assert ip.tolist() == [[22, 18]]
    pos, ip = orc.refine_positions_step(np.array([[0.5, 49.5]]), np.array([[-3.0, 3.0]]), 0.5, 2.0, 50, 49)
    assert pos.tolist() == [[0.0, 49.0]] and ip.tolist() == [[0, 49]]
    pos, ip = orc.refine_positions_step(np.array([[10.25, 11.25]]), np.array([[0.25, 0.25]]), 1.0, 2.0, 50, 50)
    assert ip.tolist() == [[10, 12]]  # 10.5 -> 10, 11.5 -> 12


def test_accumulate_shifts_matches_the_oracle(lib):
    """ptx_accumulate_shifts (library host code, no GPU) equals the oracle's step
    bit for bit over several steps of random shifts, and reports the moves."""
    from oracle import ptycho as orc
    rng = np.random.default_rng(5)
    J, max_row, max_col = 300, 90, 70
    pos_f = np.ascontiguousarray(np.stack([rng.uniform(0, max_row, J), rng.uniform(0, max_col, J)], 1))
    pos_f[:5] = [[0, 0], [max_row, max_col], [0.5, 1.5], [2.5, 3.5], [45.0, 35.0]]
    ref_f = pos_f.copy()
    ipos = np.ascontiguousarray(np.rint(pos_f).astype(np.int32))
    for it in range(4):
        shifts = np.ascontiguousarray((rng.standard_normal((J, 2)) * 1.5).astype(np.float32))
        shifts[:3] = [[-4, -4], [4, 4], [0, 0]]
        step, max_shift = 0.7, 2.0
        before = ipos.copy()
        moved = ctypes.c_int32()
        st = lib.ptx_accumulate_shifts(J, ctypes.c_void_p(shifts.ctypes.data), ctypes.c_double(step),
                                       ctypes.c_double(max_shift), max_row, max_col,
                                       ctypes.c_void_p(pos_f.ctypes.data), ctypes.c_void_p(ipos.ctypes.data),
                                       ctypes.byref(moved))
        assert st == 0
        ref_f, ref_i = orc.refine_positions_step(ref_f, shifts, step, max_shift, max_row, max_col)
        assert np.array_equal(pos_f, ref_f)
        assert np.array_equal(ipos, ref_i)
        assert moved.value == int(np.any(ipos != before, axis=1).sum())
    assert lib.ptx_accumulate_shifts(-1, None, ctypes.c_double(1.0), ctypes.c_double(1.0), 1, 1, None, None,
                                     ctypes.byref(moved)) == 1


def test_every_parameter_name_is_documented_and_checked(lib):
    """Every name ptx_set_param accepts is documented in include/ptycho.h, and
    a call without a handle is refused on the host."""
    from paper_2008_11511_gb300._lib import STATUS_NAMES
    api = open(os.path.join(ROOT, "paper_2008_11511_gb300", "csrc", "api.cu")).read()
    names = re.findall(r'strcmp\(name, "([a-z_0-9]+)"\)', api)
    header = open(HEADER).read()
    assert len(names) >= 12
    missing = [n for n in names if f'"{n}"' not in header]
    assert not missing, missing
    assert STATUS_NAMES[lib.ptx_set_param(None, b"lanes", ctypes.c_double(2.0))] == "PTX_ERR_INVALID_ARG"
