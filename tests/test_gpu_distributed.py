"""The synchronous data-parallel split on the GPU (paper Section 4's multi-GPU
setting, in its synchronous form): two gloo ranks in separate processes share
the one GPU, each holding a Ptycho of its own frames (``split_positions``).
Every cycle each rank runs its frames' passes without the overlap update, the
probe and object accumulators and the LLK are summed over the ranks by
all-reduces, and every rank normalises the same sums.  Three DM cycles and one
AP cycle must give, on both ranks, the object, probe and global per-cycle LLK
of the unsplit FP64 oracle within the single-cycle tolerance.

The ranks' kernels never wait on one another: the only exchange is the
host-side gloo all-reduce between cycles.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, d, cfg, J, over):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    from paper_2008_11511_gb300 import Ptycho
    from paper_2008_11511_gb300.distributed import ap_cycles_data_parallel, dm_cycles_data_parallel, split_positions
    from synthetic import make_config

    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = make_config(cfg, J=J, **over)
    o0 = np.load(os.path.join(d, "o0.npy"))
    p0 = np.load(os.path.join(d, "p0.npy"))
    mine = split_positions(s.positions, world, rank)
    dev = torch.device("cuda", 0)
    pb = Ptycho(torch.tensor(o0, device=dev), torch.tensor(p0, device=dev),
                torch.tensor(np.ascontiguousarray(s.iobs[mine]), device=dev), s.positions[mine], s.mask,
                with_psi=True)
    l_dm = dm_cycles_data_parallel(pb, 3, init_psi=True).cpu().numpy()
    l_ap = ap_cycles_data_parallel(pb, 1).cpu().numpy()
    torch.cuda.synchronize()
    np.save(os.path.join(d, f"obj{rank}.npy"), pb.obj.cpu().numpy())
    np.save(os.path.join(d, f"probe{rank}.npy"), pb.probe.cpu().numpy())
    np.save(os.path.join(d, f"llk{rank}.npy"), np.concatenate([l_dm, l_ap]))
    np.save(os.path.join(d, f"mine{rank}.npy"), mine)
    pb.close()
    dist.destroy_process_group()


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("cfg,J,over", [("ap64", 100, {}), ("dm256", 60, {"Ho": 512, "Wo": 512})])
def test_data_parallel_split_on_gpu_equals_unsplit_oracle(cfg, J, over):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import torch.multiprocessing as mp

    import oracle
    from paper_2008_11511_gb300 import build as b
    from synthetic import make_config
    b.build()
    s = make_config(cfg, J=J, **over)
    data = oracle.Data.make(s.iobs, s.positions, s.mask)
    # common start: the oracle's state after one AP cycle
    o0, p0, _ = oracle.ap_cycle(s.obj0, s.probe0, data)
    o0, p0 = o0.astype(np.complex64), p0.astype(np.complex64)
    world = 2
    with tempfile.TemporaryDirectory() as d:
        np.save(os.path.join(d, "o0.npy"), o0)
        np.save(os.path.join(d, "p0.npy"), p0)
        mp.start_processes(_worker, args=(world, _free_port(), d, cfg, J, over), nprocs=world, join=True,
                           start_method="spawn")
        res = [(np.load(os.path.join(d, f"obj{r}.npy")), np.load(os.path.join(d, f"probe{r}.npy")),
                np.load(os.path.join(d, f"llk{r}.npy")), np.load(os.path.join(d, f"mine{r}.npy")))
               for r in range(world)]
    # the ranks own disjoint frames that cover the scan
    assert sorted(np.concatenate([r[3] for r in res]).tolist()) == list(range(s.J))
    o, p, psi, llk_dm = oracle.cycles("DM", o0, p0, data, 3)
    o, p, l_ap = oracle.ap_cycle(o, p, data)
    ref_llk = np.array(llk_dm + [l_ap])
    d_o = oracle.object_denominator(p, s.positions, (s.Ho, s.Wo))
    ill = d_o > 1e-3 * d_o.max()
    for og, pg, lg, _ in res:
        assert rel(og[ill], o[ill]) < TOL and rel(pg, p) < TOL
        np.testing.assert_allclose(lg, ref_llk, rtol=TOL)
    # both ranks normalise the same sums: identical object and probe
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
