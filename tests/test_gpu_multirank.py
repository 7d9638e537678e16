"""The sharded outer loop through the CUDA library: two gloo ranks, each with its own process
and context on the one GPU here, split the shots, and esi_invert's reduce callback sums the
objective and the model gradient over the ranks in rank order (shard.reduce_objective).  The
ranks' kernels never wait on one another (the only exchange is the host-side sum between
evaluations), so sharing a GPU changes nothing but their speed.  Both ranks must end on the
same model, and that model must equal the single-process inversion over all shots."""
import os
import socket

import numpy as np
import pytest

from paper_2211_06300_gb300 import shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
pytestmark = pytest.mark.gpu

KW = dict(n_outer=3, n_cg=10, beta0=0.1, vmin=1400.0, vmax=2600.0)


def _problem():
    import oracle
    from oracle import outer
    from paper_2211_06300_gb300 import synth
    shape, dx, dt, nt, nb, ns = (14, 36), 10.0, 1e-3, 40, 4, 3
    v = synth.dipping_layers(shape, dx, 5, nlayers=3, vmin=1500, vmax=2300, nanom=1, sigma=25.0)
    vt = v + synth.gaussian_blob(shape, dx, 3, amp=60.0, sigma=30.0)
    rx = [np.arange(5.0, 355.0, 10.0), np.arange(0.0, 350.0, 23.0), np.array([347.5])]
    geom = synth.surface_line(ns, [55.0, 175.5, 300.0], 40.0, rx, 40.0)
    f = synth.ricker(nt, dt, 45.0)
    o_true = oracle.Oracle(vt, dx, dt, nt, nb, vref=2500.0)
    d = [o_true.forward(o_true.shot(geom.src_xyz[s], geom.receivers(s)), wavelet=f)["traces"]
         for s in range(ns)]
    pb = outer.Problem(dx, dt, nt, nb, 2500.0, [geom.src_xyz[s] for s in range(ns)],
                       [geom.receivers(s) for s in range(ns)], d, wavelets=[f] * ns)
    return v, geom, pb


def _invert(shots, reduce=None):
    from paper_2211_06300_gb300 import esi
    v, geom, pb = _problem()
    sub = geom.select(list(shots))
    f64 = torch.float64
    ctx = esi.Context(torch.tensor(v, dtype=f64, device="cuda"), pb.dx, pb.dt, pb.nt, pb.nb,
                      sub, vref=pb.vref)
    d = torch.tensor(np.concatenate([pb.d[s].ravel() for s in shots]), dtype=f64, device="cuda")
    vel = torch.tensor(v, dtype=f64, device="cuda")
    _, rep = ctx.invert(d, vel, reduce=reduce, **KW)
    ctx.close()
    return vel.cpu().numpy(), rep


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.shot_range(3, rank, world)

        def red(J, g):   # the library's gradient on the device, summed over ranks on the host
            gc = g.cpu()
            Jt = shard.reduce_objective(J, gc, dist)
            g.copy_(gc)
            return Jt
        vel, rep = _invert(range(lo, hi), red)
        np.save(os.path.join(out, f"r{rank}.npy"),
                np.concatenate([vel.ravel(), rep["J_end"], [rep["evaluations"]]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_of_the_library_reproduce_the_single_process_inversion(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)                    # every rank ends on the same model
    vel, rep = _invert(range(3))
    ref = np.concatenate([vel.ravel(), rep["J_end"], [rep["evaluations"]]])
    assert r0.shape == ref.shape and r0[-1] == ref[-1] > 3
    v0 = _problem()[0].ravel()
    n = v0.size
    # the shots' partial sums are added in the same order as in one process: FP64 rounding
    assert np.linalg.norm(r0[:n] - ref[:n]) <= 1e-12 * np.linalg.norm(ref[:n] - v0)
    assert np.allclose(r0[n:-1], ref[n:-1], rtol=1e-12, atol=0)
