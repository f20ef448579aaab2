"""The time-slab decomposition of the search and the vote, run by gloo ranks
on the CPU with the oracle as each rank's arithmetic: rank r owns the
targets and occluded voxels of frames [r T / n, (r + 1) T / n). After every
Jacobi iteration a rank takes from the others only the shifts of the frame
on each side of its slab; after the search, the shifts and distances of the
two frames on each side; after the vote, the occluded voxels of the other
slabs. The assembled shifts, distances, voxels and evaluation count equal
the single-process oracle's bit for bit (the change sums, added in another
order, to rounding). This is the exchange plan the library's time slabs
(vi_run_slabs) follow between contexts."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1503_05528_gb300 import synth

N_PM = 4
KEY = (17, 5)
TAG = O.tag(O.PURPOSE_SEARCH, 0, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _state():
    clip = synth.small_layered(W=40, H=32, T=12, levels=1, seed=1801)
    lv = O.build_pyramid(clip.rgb, clip.mask, 1, True)[0]
    rng = np.random.default_rng(3)
    x = lv.x.copy()
    h = lv.hole.astype(bool)
    x[h] = rng.random((int(h.sum()), x.shape[-1]), dtype=np.float32) * np.float32(0.8) + np.float32(0.1)
    phi = O.init_nnf(lv.htilde, lv.dtilde, KEY, O.tag(O.PURPOSE_INIT, 0))
    return lv, np.ascontiguousarray(x), phi


def _slab(r, n, T):
    return r * T // n, (r + 1) * T // n


def _owner(t, n, T):
    return next(r for r in range(n) if t < _slab(r, n, T)[1])


def _gather(a):
    parts = [torch.empty_like(torch.from_numpy(a)) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, torch.from_numpy(np.ascontiguousarray(a)))
    return [p.numpy() for p in parts]


def _halo(arrays, r, n, T, w):
    """Frames within w of slab r taken from their owners (every array is
    gathered; only the halo frames are used)."""
    t0, t1 = _slab(r, n, T)
    for a in arrays:
        got = _gather(a)   # every rank gathers, so the collective matches across ranks
        for t in list(range(max(t0 - w, 0), t0)) + list(range(t1, min(t1 + w, T))):
            a[t] = got[_owner(t, n, T)][t]


def _worker(rank, world, port, out, w_sweep=1, w_vote=2):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lv, x, phi = _state()
        T = x.shape[0]
        t0, t1 = _slab(rank, world, T)
        frames = np.zeros(lv.hole.shape, bool)
        frames[t0:t1] = True
        own_t = (lv.htilde.astype(bool) & frames).astype(np.uint8)
        own_h = (lv.hole.astype(bool) & frames).astype(np.uint8)
        d2 = np.full(lv.hole.shape, np.inf, np.float32)
        evals = O.rescore(x, own_t, lv.dtilde, phi, d2)
        for k in range(1, N_PM + 1):
            evals += O.ann_iteration(x, lv.htilde, lv.dtilde, phi, d2, k, key=KEY, tag_base=TAG, own=own_t)
            _halo([phi], rank, world, T, w_sweep)    # propagation in t reads t -+ 1
        _halo([phi, d2], rank, world, T, w_vote)     # the vote reads patches two frames away
        xv, ch = O.vote(x, own_h, lv.htilde, phi, d2, weighted=True)
        # assemble: every rank's own targets and occluded voxels
        phis, d2s, xs = _gather(phi), _gather(d2), _gather(xv)
        ev = torch.tensor([evals], dtype=torch.int64)
        dist.all_reduce(ev)
        chs = torch.tensor([ch], dtype=torch.float64)
        dist.all_reduce(chs)
        if rank == 0:
            P, D, X = phis[0].copy(), d2s[0].copy(), xs[0].copy()
            for r in range(1, world):
                a, b = _slab(r, world, T)
                m = np.zeros(lv.hole.shape, bool)
                m[a:b] = True
                P[m], D[m], X[m] = phis[r][m], d2s[r][m], xs[r][m]
            out["res"] = (P, D, X, int(ev.item()), float(chs.item()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_equal_the_single_process_oracle(world):
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    P, D, X, evals, change = out["res"]
    lv, x, phi = _state()
    d2 = np.full(lv.hole.shape, np.inf, np.float32)
    e_ref = O.ann(x, lv.htilde, lv.dtilde, phi, d2, n_pm=N_PM, schedule="JAC", key=KEY, tag_base=TAG)
    x_ref, ch_ref = O.vote(x, lv.hole, lv.htilde, phi, d2, weighted=True)
    t = lv.htilde == 1
    np.testing.assert_array_equal(P[t], phi[t])
    np.testing.assert_array_equal(D[t].view(np.uint32), d2[t].view(np.uint32))
    h = lv.hole == 1
    np.testing.assert_array_equal(X[h].view(np.uint32), x_ref[h].view(np.uint32))
    assert evals == e_ref
    assert abs(change - ch_ref) <= 1e-12 * max(abs(ch_ref), 1.0)


def test_without_the_halo_the_slabs_disagree():
    # control: with no frames exchanged the slabs' search and vote differ
    # from the single-process oracle, so the test above checks the exchange
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, _free_port(), out, 0, 0), nprocs=2, join=True)
    P, D, X, evals, change = out["res"]
    lv, x, phi = _state()
    d2 = np.full(lv.hole.shape, np.inf, np.float32)
    O.ann(x, lv.htilde, lv.dtilde, phi, d2, n_pm=N_PM, schedule="JAC", key=KEY, tag_base=TAG)
    t = lv.htilde == 1
    assert not np.array_equal(P[t], phi[t])
