"""Split (partitioned) domains on the CPU (Section 2.2: the sparse domain is decomposed
over ranks, every step ends with a non-blocking exchange of the populations that cross
the cuts, and only averaged values are gathered for the iolets; Section 2.2.1: the cut
balances the work).

  * the C++ planner's cut, ghost counts and halo matrix against a restatement in
    Python on the oracle's neighbour table (equal site counts; and a weighted cut whose
    partition costs differ by at most one site's weight);
  * the oracle itself run on two gloo ranks, each stepping only its own contiguous range
    of the canonical site list plus ghost copies of the sites it pulls from, the halo
    values exchanged by non-blocking send/recv after every step and the per-site
    moments gathered to rank 0 for the iolet means: the final state and means are
    bit-identical to the unpartitioned oracle.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest

from paper_2010_04144_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STEPS = 60


def _geo():
    return S.tree(S.TreeSpec(depth=3, root_radius=5, seed=3), inlet_speed=0.04, period=40.0)


def _layout_ref(nbr, n, k, weights):
    pre = np.concatenate([[0.0], np.cumsum(weights)])
    first = [0]
    for p in range(1, k):
        c = int(np.searchsorted(pre, pre[n] * p / k, side="left"))
        c = min(max(c, first[-1] + 1), n - (k - p))
        first.append(c)
    first.append(n)
    ghosts, halo = [], np.zeros((k, k), np.int64)
    for p in range(k):
        a, b = first[p], first[p + 1]
        rows = nbr[:, a:b]
        pulls = rows[(rows >= 0) & ((rows < a) | (rows >= b))]
        ghosts.append(len(np.unique(pulls)))
        owner = np.searchsorted(first, pulls, side="right") - 1
        for q in owner:
            halo[q, p] += 1
    return np.array(first), np.array(ghosts), halo


@pytest.mark.parametrize("k,bw", [(1, 1.0), (2, 1.0), (3, 1.0), (7, 1.0), (4, 6.0)])
def test_split_layout_matches_restatement(hemegb_lib, oracle_mod, k, bw):
    geo = S.tree(S.TreeSpec(depth=4, root_radius=6, seed=7))
    od = oracle_mod.Domain(geo.xyz, geo.iolets, tau=0.8)
    boundary = (od.nbr < -1).any(axis=0)
    w = np.where(boundary, bw, 1.0)
    first, ghosts, halo = hemegb_lib.split_layout(geo.xyz, geo.iolets, k, boundary_weight=bw)
    rf, rg, rh = _layout_ref(od.nbr, od.n, k, w)
    assert np.array_equal(first, rf) and np.array_equal(ghosts, rg) and np.array_equal(halo, rh)
    cost = [w[first[p]:first[p + 1]].sum() for p in range(k)]
    assert max(cost) - min(cost) <= 2 * bw
    assert np.all(np.diag(halo) == 0)
    if k > 1:
        assert halo.sum() > 0 and np.all(ghosts > 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, ws, port, q):
    """One rank of the partitioned oracle: owned range + ghosts, halo by isend/irecv."""
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    geo = _geo()
    full = oracle.Domain(geo.xyz, geo.iolets, tau=0.8)      # the global table is set-up input
    n = full.n
    first = [math.ceil(n * p / ws) for p in range(ws)] + [n]
    a, b = first[rank], first[rank + 1]
    own = np.arange(a, b)
    rows = full.nbr[:, a:b]
    ghosts = np.unique(rows[(rows >= 0) & ((rows < a) | (rows >= b))])
    loc_sites = np.concatenate([own, ghosts])
    n_own, n_loc = b - a, loc_sites.size
    local = {int(g): n_own + j for j, g in enumerate(ghosts)}
    nbr = np.full((18, n_loc), -1, np.int32)                  # ghost rows: walls (never used)
    for i in range(18):
        for s in range(n_own):
            v = int(rows[i, s])
            nbr[i, s] = (v - a) if a <= v < b else (local[v] if v >= 0 else v)
    part = oracle.Domain.__new__(oracle.Domain)               # a local view with the same arithmetic
    part.n, part.iolets, part.tau, part._io = n_loc, full.iolets, full.tau, full._io
    part.xyz = np.ascontiguousarray(full.xyz[loc_sites])
    part.nbr = nbr
    F = np.zeros((19, n_loc))
    buf = np.zeros_like(F)
    mom = np.zeros((n_loc, 4))
    # halo: what each peer needs from me (direction I, my local index), and where I put
    # what I receive from each peer (direction I, ghost local index), canonical order
    owner = lambda v: int(np.searchsorted(first, v, side="right") - 1)
    recv_from = {}
    for i in range(18):
        for s in range(n_own):
            v = int(rows[i, s])
            if v >= 0 and not (a <= v < b):
                recv_from.setdefault(owner(v), []).append((i + 1, v))
    for key in recv_from:
        recv_from[key].sort(key=lambda e: (e[1], e[0]))
    # exchange the request lists once (set-up), then values every step
    send_to = {}
    for peer in range(ws):
        if peer == rank:
            continue
        mine = recv_from.get(peer, [])
        lst = [None]
        if rank < peer:
            dist.send_object_list([mine], dst=peer)
            dist.recv_object_list(lst, src=peer)
        else:
            dist.recv_object_list(lst, src=peer)
            dist.send_object_list([mine], dst=peer)
        send_to[peer] = [(I, v - a) for I, v in lst[0]]
    io = full.iolets

    def bc(t):
        return np.array([x.value * oracle.pulse(x.pulse, t, x.period) for x in io])

    adj = (full.nbr < -1).any(axis=0)
    for t in range(1, STEPS + 1):
        part.step_into(F, buf, bc(t), mom)
        F, buf = buf, F
        reqs, inbox = [], {}
        for peer, lst in send_to.items():
            vals = torch.tensor([F[I, s] for I, s in lst], dtype=torch.float64)
            reqs.append(dist.isend(vals, dst=peer))
        for peer, lst in recv_from.items():
            inbox[peer] = torch.zeros(len(lst), dtype=torch.float64)
            reqs.append(dist.irecv(inbox[peer], src=peer))
        for r in reqs:
            r.wait()
        for peer, lst in recv_from.items():
            for (I, v), x in zip(lst, inbox[peer].numpy()):
                F[I, local[v]] = x
        # iolet means: the adjacent sites' moments gathered to rank 0 (canonical order)
        sel = np.nonzero(adj[a:b])[0]
        got = [None] * ws if rank == 0 else None
        dist.gather_object((a + sel, mom[sel]), got, dst=0)
        if rank == 0:
            M_full = np.zeros((n, 4))
            for idx, m in got:
                M_full[idx] = m
            M = full.iolet_means(M_full)
    out = [None] * ws if rank == 0 else None
    dist.gather_object((a, F[:, :n_own].copy()), out, dst=0)
    if rank == 0:
        Fg = np.zeros((19, n))
        for a0, Fp in out:
            Fg[:, a0:a0 + Fp.shape[1]] = Fp
        q.put((Fg, M))
    dist.barrier()
    dist.destroy_process_group()


def test_partitioned_oracle_gloo_bit_identical(oracle_mod):
    import torch.multiprocessing as mp

    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    Fg, M = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    geo = _geo()
    od = oracle_mod.Domain(geo.xyz, geo.iolets, tau=0.8)
    sysm = oracle_mod.System([od])
    sysm.step(STEPS)
    assert np.array_equal(Fg, od.F)
    assert np.array_equal(M, sysm.M[0])
    assert np.abs(od.F).max() > 0
