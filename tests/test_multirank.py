"""The N > 1 path on CPU: two gloo ranks split the shots, each computes its shots' misfit
gradients with the oracle, and the ordered sum over ranks equals the single-process sum over
all shots (the one exchange of the outer loop); times reduce by max, work by sum.  The whole
outer loop (Algorithm "nestedloop") sharded the same way reproduces the single-process
inversion."""
import os
import socket

import numpy as np
import pytest

from paper_2211_06300_gb300 import shard

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def test_shot_range_partitions_every_shot_once():
    for ns in (1, 5, 16, 17, 64):
        for world in (1, 2, 3, 4, 8):
            got = []
            for r in range(world):
                lo, hi = shard.shot_range(ns, r, world)
                assert 0 <= lo <= hi <= ns
                got += list(range(lo, hi))
            assert got == list(range(ns))
            sizes = [np.subtract(*shard.shot_range(ns, r, world)[::-1]) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shot_range(4, 2, 2)


def _case():
    import oracle
    from paper_2211_06300_gb300 import synth
    shape, dx, dt, nt, nb = (24, 30), 10.0, 1e-3, 60, 5
    v = synth.dipping_layers(shape, dx, 3, nlayers=3, vmin=1500, vmax=2400, nanom=1, sigma=30.0)
    v0 = synth.smooth(v, 30.0, dx)
    ns = 5
    recs = [np.arange(0.0, 290.0, 20.0) for _ in range(ns)]
    geom = synth.surface_line(ns, list(np.linspace(40.0, 250.0, ns)), 30.0, recs, 20.0)
    wav = synth.ricker(nt, dt, 25.0)
    o_true = oracle.Oracle(v, dx, dt, nt, nb)
    o = oracle.Oracle(v0, dx, dt, nt, nb, vref=float(v.max()))
    return o_true, o, geom, wav, ns


def _partial(lo, hi):
    o_true, o, geom, wav, _ = _case()
    g = np.zeros(o.N)
    J = 0.0
    for s in range(lo, hi):
        sh_t = o_true.shot(geom.src_xyz[s], geom.receivers(s))
        sh = o.shot(geom.src_xyz[s], geom.receivers(s))
        d = o_true.forward(sh_t, wavelet=wav)["traces"]
        j, gs = o.misfit_gradient(sh, d, wavelet=wav, param="v")
        g += gs
        J += j
    return J, g


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ns = 5
        lo, hi = shard.shot_range(ns, rank, world)
        J, g = _partial(lo, hi)
        t = torch.tensor(np.concatenate([[J], g]), dtype=torch.float64)
        tot = shard.ordered_sum(t, dist)
        tmax = shard.max_over_ranks(1.0 + rank, dist)
        work = shard.sum_over_ranks(hi - lo, dist)
        np.save(os.path.join(out, f"r{rank}.npy"), np.concatenate([tot.numpy(), [tmax, work]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reproduce_the_single_process_gradient(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert np.array_equal(r0, r1)                  # identical on every rank
    J, g = _partial(0, 5)
    ref = np.concatenate([[J], g])
    assert np.allclose(r0[:-2], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    assert r0[-2] == 2.0 and r0[-1] == 5.0          # max time, total shots


def _outer_case():
    import oracle
    from oracle import outer
    from paper_2211_06300_gb300 import synth
    shape, dx, dt, nt, nb = (14, 16), 10.0, 1e-3, 30, 4
    v = synth.dipping_layers(shape, dx, 5, nlayers=3, vmin=1500, vmax=2300, nanom=1, sigma=25.0)
    vt = v + synth.gaussian_blob(shape, dx, 3, amp=60.0, sigma=30.0)
    srcs = [(25.0, 0.0, 40.0), (75.0, 0.0, 40.0), (125.0, 0.0, 40.0)]
    recs = [np.array([(x, 0.0, 40.0) for x in np.arange(5.0, 155.0, 10.0)])] * 3
    f = synth.ricker(nt, dt, 45.0)
    o_true = oracle.Oracle(vt, dx, dt, nt, nb, vref=2500.0)
    d = [o_true.forward(o_true.shot(s, r), wavelet=f)["traces"] for s, r in zip(srcs, recs)]
    pb = outer.Problem(dx, dt, nt, nb, 2500.0, srcs, recs, d, wavelets=[f] * 3)
    opt = outer.Options(mode="esi", n_outer=3, n_cg=10, beta0=0.1, vmin=1400, vmax=2600)
    return v, pb, opt


def _outer_rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import outer
        v, pb, opt = _outer_case()
        lo, hi = shard.shot_range(len(pb.src_xyz), rank, world)
        h = outer.invert(v, pb, opt, reduce=lambda J, g: shard.reduce_objective(J, g, dist),
                         shots=range(lo, hi))
        np.save(os.path.join(out, f"o{rank}.npy"),
                np.concatenate([h["v"].ravel(), h["J_end"], [len(h["J_end"])]]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_outer_loop(tmp_path):
    import torch.multiprocessing as mp
    from oracle import outer
    world = 2
    mp.start_processes(_outer_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    r0 = np.load(tmp_path / "o0.npy")
    r1 = np.load(tmp_path / "o1.npy")
    assert np.array_equal(r0, r1)
    v, pb, opt = _outer_case()
    h = outer.invert(v, pb, opt)
    ref = np.concatenate([h["v"].ravel(), h["J_end"], [len(h["J_end"])]])
    assert r0.shape == ref.shape
    assert np.allclose(r0, ref, rtol=1e-10, atol=0)
