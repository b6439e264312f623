"""Data-parallel split over ranks, on CPU with the gloo backend (world size 2 and 3).

Each rank computes the Psi2ObjProbe numerators/denominators of its share of
the frames (with the FP64 oracle standing in for the GPU cycle), the packed
accumulators are summed with paper_2008_11511_gb300.distributed's all-reduce,
and the normalised object and probe must equal the unsplit cycle.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _pack(sums, Ho, Wo, K, N):
    n_o, d_o, n_p, d_p = sums
    ao = np.zeros((Ho, Wo, 4))
    ao[..., 0], ao[..., 1], ao[..., 2] = n_o.real, n_o.imag, d_o
    ap = np.zeros((K, N, N, 4))
    ap[..., 0], ap[..., 1], ap[..., 2] = n_p.real, n_p.imag, d_p[None]
    return torch.from_numpy(ao), torch.from_numpy(ap)


def _worker(rank, world, port, outdir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import oracle
    from paper_2008_11511_gb300.distributed import allreduce_accumulators, split_positions
    from synthetic import make_config

    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = make_config("ap64", J=40)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    mine = split_positions(s.positions, world, rank)
    obj = s.obj0.astype(np.complex128)
    probe = s.probe0.astype(np.complex128)
    # this rank's AP cycle contribution
    phi_hat = oracle.ft(oracle.obj_probe_to_psi(obj, probe, data.positions[mine]))
    llk = torch.tensor([oracle.llk_poisson(oracle.calc_intensity(phi_hat), data.iobs[mine], data.mask)],
                       dtype=torch.float64)
    psi = oracle.ift(oracle.apply_amplitude(phi_hat, data.iobs[mine], data.mask))
    # probe sums of this rank's frames -> all-reduce -> probe update
    n_p, d_p = oracle.psi_to_probe_sums(psi, obj, data.positions[mine])
    _, ap = _pack((np.zeros(obj.shape, complex), np.zeros(obj.shape), n_p, d_p), s.Ho, s.Wo, s.K, s.N)
    allreduce_accumulators(None, ap, llk)
    p = ap.numpy()
    p1 = oracle.inertia_update(probe, p[..., 0] + 1j * p[..., 1], p[0, ..., 2][None], 1e-2)
    # object sums with the new probe -> all-reduce -> object update
    n_o, d_o = oracle.psi_to_obj_sums(psi, p1, data.positions[mine], obj.shape)
    ao, _ = _pack((n_o, d_o, np.zeros_like(probe), np.zeros(probe.shape[1:])), s.Ho, s.Wo, s.K, s.N)
    allreduce_accumulators(ao, None)
    a = ao.numpy()
    o1 = oracle.inertia_update(obj, a[..., 0] + 1j * a[..., 1], a[..., 2], 1e-2)
    np.save(os.path.join(outdir, f"obj{rank}.npy"), o1)
    np.save(os.path.join(outdir, f"probe{rank}.npy"), p1)
    np.save(os.path.join(outdir, f"llk{rank}.npy"), llk.numpy())
    np.save(os.path.join(outdir, f"mine{rank}.npy"), mine)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_cycle_equals_unsplit(world):
    import torch.multiprocessing as mp

    import oracle
    from synthetic import make_config
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, _free_port(), d), nprocs=world, join=True)
        s = make_config("ap64", J=40)
        data = oracle.Data.make(s.iobs, s.positions, s.mask)
        o_ref, p_ref, l_ref = oracle.ap_cycle(s.obj0, s.probe0, data)
        owned = np.concatenate([np.load(os.path.join(d, f"mine{r}.npy")) for r in range(world)])
        assert np.array_equal(np.sort(owned), np.arange(s.J))  # every frame on exactly one rank
        for r in range(world):
            o = np.load(os.path.join(d, f"obj{r}.npy"))
            p = np.load(os.path.join(d, f"probe{r}.npy"))
            l = float(np.load(os.path.join(d, f"llk{r}.npy"))[0])
            assert np.linalg.norm(o - o_ref) / np.linalg.norm(o_ref) < 1e-12
            assert np.linalg.norm(p - p_ref) / np.linalg.norm(p_ref) < 1e-12
            assert abs(l - l_ref) < 1e-9 * abs(l_ref)


def test_split_positions_is_a_spatial_partition():
    from paper_2008_11511_gb300.distributed import split_positions
    rng = np.random.default_rng(0)
    pos = rng.integers(0, 1000, size=(101, 2))
    parts = [split_positions(pos, 4, r) for r in range(4)]
    assert sorted(np.concatenate(parts).tolist()) == list(range(101))
    assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    rows = [pos[p, 0] for p in parts]
    for a, b in zip(rows[:-1], rows[1:]):
        assert a.max() <= b.min()
