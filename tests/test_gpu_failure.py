"""Failure detection without a GPU fault.

The library's device-side waits (tensor-copy arrivals in the object gather and
the column pass, MMA commits in the tensor-core column pass) are bounded: a
wait that runs out records the fact in the handle's error flag (mapped host
memory) and the kernel returns, so the context stays usable, and the next
cycle call reports PTX_ERR_TIMEOUT once.  Here the waits that run out are
ptx_wait_selftest's, on a flag that nothing sets, and a tensor-core stage's,
on an mbarrier whose commit is never issued (with no MMA in flight); no GPU
fault, trap or hang is involved.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synthetic import make_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2008_11511_gb300 import build as b
    b.build()


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), device="cuda")


def _rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def test_wait_timeout_is_reported_once_and_the_handle_stays_usable():
    from paper_2008_11511_gb300 import Ptycho, _lib
    from paper_2008_11511_gb300._lib import PtychoError
    s = make_config("ap64", J=30)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = Ptycho(_dev(o0), _dev(p0), _dev(s.iobs), s.positions, s.mask)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.call("ptx_wait_selftest", pb._handle(), 2000, stream)  # gives up after 2 ms
    torch.cuda.synchronize()
    with pytest.raises(PtychoError) as ei:
        pb.ap(1)
    assert ei.value.status_name == "PTX_ERR_TIMEOUT"
    assert "bounded device wait" in str(ei.value)
    # reported once; the refused call enqueued nothing, so the next cycle starts from (o0, p0)
    llk = pb.ap(1).cpu().numpy()
    o, p, l = oracle.ap_cycle(o0, p0, data)
    assert _rel(pb.probe.cpu().numpy(), p) < 1e-5
    d = oracle.object_denominator(p, s.positions, o.shape)
    ill = d > 1e-3 * d.max()
    assert _rel(pb.obj.cpu().numpy()[ill], o[ill]) < 1e-5
    assert abs(llk[0] - l) < 1e-5 * abs(l)
    pb.close()


def test_wait_selftest_rejects_limits_out_of_range():
    from paper_2008_11511_gb300 import Ptycho, _lib
    from paper_2008_11511_gb300._lib import PtychoError
    s = make_config("ap64", J=10)
    pb = Ptycho(_dev(s.obj0), _dev(s.probe0), _dev(s.iobs), s.positions, s.mask)
    for bad in (0, -5, 1000001):
        with pytest.raises(PtychoError) as ei:
            _lib.call("ptx_wait_selftest", pb._handle(), bad, None)
        assert ei.value.status_name == "PTX_ERR_INVALID_ARG"
    pb.ap(1)  # nothing was enqueued; the handle works
    pb.close()


def test_counts_to_float_is_exact_with_a_ragged_tail():
    """uint16 photon counts widened on the device: every value exact, n not a
    multiple of the 8 counts a thread converts at once."""
    from paper_2008_11511_gb300 import counts_to_float
    rng = np.random.default_rng(9)
    n = 1_000_003
    c = rng.integers(0, 65536, size=n, dtype=np.uint16)
    c[:3] = (0, 65535, 1)
    dst = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    counts_to_float(dst, torch.from_numpy(c).cuda())
    assert np.array_equal(dst.cpu().numpy(), c.astype(np.float32))


def test_counts_to_float_rejects_misaligned_pointers():
    from paper_2008_11511_gb300 import _lib
    from paper_2008_11511_gb300._lib import PtychoError
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    src = torch.zeros(64, dtype=torch.uint16, device="cuda")
    with pytest.raises(PtychoError) as ei:
        _lib.call("ptx_counts_to_float", ctypes.c_void_p(buf.data_ptr() + 4), ctypes.c_void_p(src.data_ptr()),
                  ctypes.c_size_t(8), None)
    assert ei.value.status_name == "PTX_ERR_INVALID_ARG"


def test_tensor_core_stage_wait_gives_up_and_reports():
    """A tensor-core stage whose MMAs and commit are never issued (the
    "tc_selftest" switch) makes its half's bounded mbarrier wait run out while
    every other half of the launch completes normally: the next call reports
    PTX_ERR_TIMEOUT once, and the handle then runs cycles that match the oracle."""
    from paper_2008_11511_gb300 import Ptycho, PtychoError
    s = make_config("dm256", J=24, Ho=512, Wo=512)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    pb = Ptycho(torch.tensor(o0, device="cuda"), torch.tensor(p0, device="cuda"),
                torch.tensor(s.iobs, device="cuda"), s.positions, s.mask)
    pb.set_param("tc", 1)
    pb.set_param("tc_selftest", 1)
    pb.ap(1)
    torch.cuda.synchronize()
    with pytest.raises(PtychoError, match="TIMEOUT"):
        pb.ap(1)
    pb.set_param("tc_selftest", 0)
    pb.obj.copy_(torch.tensor(o0, device="cuda"))
    pb.probe.copy_(torch.tensor(p0, device="cuda"))
    pb.ap(1)
    o, p, _ = oracle.ap_cycle(o0, p0, data)
    d = oracle.object_denominator(p, s.positions, (s.Ho, s.Wo))
    ill = d > 1e-3 * d.max()
    obj = pb.obj.cpu().numpy()
    assert np.linalg.norm(obj[ill] - o[ill]) / np.linalg.norm(o[ill]) < 2e-5
    assert np.linalg.norm(pb.probe.cpu().numpy() - p) / np.linalg.norm(p) < 2e-5
    pb.close()


def test_counts8_round_trip_is_exact_with_a_ragged_tail():
    """The one-byte count form: host encoding, device decoding (uint8 widened,
    then the escapes written over them) restores every count exactly; n not a
    multiple of the 16 counts a thread converts at once; also without escapes."""
    from paper_2008_11511_gb300 import counts8_to_float, encode_counts8
    rng = np.random.default_rng(11)
    n = 1_000_003
    c = rng.poisson(40.0, size=n).astype(np.uint16)
    hot = rng.choice(n, size=20_000, replace=False)
    c[hot] = rng.integers(255, 65536, size=hot.size, dtype=np.uint16)
    c[:4] = (0, 254, 255, 65535)
    c[-2:] = (256, 255)
    out8, idx, val = encode_counts8(c)
    dst = torch.full((n,), -1.0, dtype=torch.float32, device="cuda")
    counts8_to_float(dst, torch.from_numpy(out8).cuda(), torch.from_numpy(idx).cuda(), torch.from_numpy(val).cuda())
    assert np.array_equal(dst.cpu().numpy(), c.astype(np.float32))
    # an escape whose index lies outside the array is skipped
    guard = torch.full((n + 16,), -1.0, dtype=torch.float32, device="cuda")
    counts8_to_float(guard[:n], torch.from_numpy(out8).cuda(),
                     torch.from_numpy(np.append(idx, np.uint32(n))).cuda(),
                     torch.from_numpy(np.append(val, np.uint16(7))).cuda())
    g = guard.cpu().numpy()
    assert np.array_equal(g[:n], c.astype(np.float32)) and np.all(g[n:] == -1.0)
    small = np.minimum(c, 200).astype(np.uint16)
    o8, i8, v8 = encode_counts8(small)
    assert i8.size == 0
    dst.fill_(-1.0)
    counts8_to_float(dst, torch.from_numpy(o8).cuda(), torch.from_numpy(i8).cuda(), torch.from_numpy(v8).cuda())
    assert np.array_equal(dst.cpu().numpy(), small.astype(np.float32))


def test_counts8_to_float_rejects_misaligned_pointers():
    from paper_2008_11511_gb300 import _lib
    from paper_2008_11511_gb300._lib import PtychoError
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    src = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(PtychoError) as ei:
        _lib.call("ptx_counts8_to_float", ctypes.c_void_p(buf.data_ptr() + 4), ctypes.c_void_p(src.data_ptr()),
                  ctypes.c_size_t(16), None, None, ctypes.c_size_t(0), None)
    assert ei.value.status_name == "PTX_ERR_INVALID_ARG"
