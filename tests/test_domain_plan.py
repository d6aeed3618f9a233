"""Host logic of the domain decomposition (no GPU): the brick partition and the
halo boxes of include/mhd.h (mhd_domain_brick, mhd_domain_halo), which the
library's pack, copy and unpack kernels follow.

  * the bricks tile the grid, their sizes differ by at most one cell;
  * every send box lies in its brick's interior, every receive box in its
    ghost shell, and the box a brick sends in direction o matches, in
    extents, the box its peer receives from direction -o;
  * packing every brick's send boxes, delivering each to its peer's receive
    box and unpacking there fills every ghost slot with the value the
    undivided grid has at that global position: its periodic wrap on
    periodic axes (the paper's exchange with 8 / 26 neighbours, §3.4,
    Fig. par_ex).  Done once with all bricks in one process, and once with
    two gloo ranks that each own a brick and exchange the packed buffers by
    send / recv."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_2511_20337_b300 import mhd
from paper_2511_20337_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    ("3d-periodic-plm", W.base_cfg(3, (9, 8, 7), (0, 0, 0), (1, 1, 1)), (2, 2, 2)),
    ("3d-periodic-wenoz", W.base_cfg(3, (9, 8, 8), (0, 0, 0), (1, 1, 1), recon="wenoz"), (2, 1, 2)),
    ("3d-outflow-x", W.base_cfg(3, (10, 6, 7), (0, 0, 0), (1, 1, 1), bc=["outflow", "outflow"] + ["periodic"] * 4),
     (3, 1, 2)),
    ("3d-outflow-all-ppm", W.base_cfg(3, (8, 9, 8), (0, 0, 0), (1, 1, 1), recon="ppm", bc="outflow"), (2, 2, 2)),
    ("2d-periodic", W.base_cfg(2, (11, 7), (0, 0), (1, 1)), (3, 2)),
    ("2d-mixed", W.base_cfg(2, (9, 10), (0, 0), (1, 1), bc=["periodic", "periodic", "outflow", "outflow", "periodic", "periodic"]), (1, 3)),
    ("3d-one-brick", W.base_cfg(3, (6, 5, 4), (0, 0, 0), (1, 1, 1)), (1, 1, 1)),
]


def G_of(cfg):
    return 2 if cfg["recon"] == "plm" else 3


def nbricks(parts):
    return int(np.prod(list(parts) + [1] * (3 - len(parts))))


def dims(cfg):
    nd = cfg["ndim"]
    return [cfg["n"][d] if d < nd else 1 for d in range(3)]


@pytest.mark.parametrize("name,cfg,parts", CASES, ids=[c[0] for c in CASES])
def test_bricks_tile_the_grid(name, cfg, parts):
    N = dims(cfg)
    cover = np.zeros(N[::-1], dtype=int)
    sizes = {d: set() for d in range(3)}
    for b in range(nbricks(parts)):
        lo, n = mhd.domain_brick(cfg, parts, b)
        cover[lo[2]:lo[2] + n[2], lo[1]:lo[1] + n[1], lo[0]:lo[0] + n[0]] += 1
        for d in range(3):
            sizes[d].add(n[d])
    assert np.all(cover == 1)
    for d in range(3):
        assert max(sizes[d]) - min(sizes[d]) <= 1


def test_bad_partitions_are_refused():
    cfg = W.base_cfg(3, (9, 8, 7), (0, 0, 0), (1, 1, 1))
    for parts in ((0, 1, 1), (5, 1, 1), (1, 1, 3), (2, 2, 3)):  # zero, bricks below G + 1 cells
        with pytest.raises(mhd.MhdError):
            mhd.domain_brick(cfg, parts, 0)
    cfg2 = W.base_cfg(2, (9, 8), (0, 0), (1, 1))
    with pytest.raises(mhd.MhdError):
        mhd.domain_brick(cfg2, (1, 1, 2), 0)      # an inactive axis split
    with pytest.raises(mhd.MhdError):
        mhd.domain_brick(dict(cfg, divb="glm"), (2, 1, 1), 0)   # CT only


@pytest.mark.parametrize("name,cfg,parts", CASES, ids=[c[0] for c in CASES])
def test_boxes_pair_up_and_stay_in_place(name, cfg, parts):
    G, nd = G_of(cfg), cfg["ndim"]
    nb = nbricks(parts)
    per = [cfg["bc"][2 * d] == "periodic" for d in range(nd)]
    send = {b: mhd.domain_halo(cfg, parts, b, True) for b in range(nb)}
    recv = {b: mhd.domain_halo(cfg, parts, b, False) for b in range(nb)}
    pp = list(parts) + [1] * (3 - len(parts))
    for b in range(nb):
        _, n = mhd.domain_brick(cfg, parts, b)
        c = (b % pp[0], (b // pp[0]) % pp[1], b // (pp[0] * pp[1]))
        # the last brick of an outflow axis also sends its slot n (the upper boundary face)
        top = [n[d] + (1 if d < nd and not per[d] and c[d] == pp[d] - 1 else 0) for d in range(3)]
        # one box per existing neighbour: 26 (8 in 2D) when every axis is periodic
        if all(per):
            assert len(send[b]) == len(recv[b]) == (26 if nd == 3 else 8)
        for boxes, is_send in ((send[b], True), (recv[b], False)):
            off = 0
            for x in boxes:
                assert x["offset"] == off
                off += int(np.prod(x["ext"]))
                for d in range(3):
                    lo, e = x["lo"][d], x["ext"][d]
                    if d >= nd:
                        assert (lo, e, x["dir"][d]) == (0, 1, 0)
                    elif is_send:
                        assert 0 <= lo and lo + e <= top[d]    # interior (and the upper boundary face)
                    else:
                        assert -G <= lo and lo + e <= n[d] + G + 1
                if not is_send:                                # at least one ghost axis
                    assert any(x["lo"][d] < 0 or x["lo"][d] >= n[d] for d in range(nd))
        for x in send[b]:
            back = [r for r in recv[x["peer"]] if r["dir"] == tuple(-o for o in x["dir"])]
            assert len(back) == 1 and back[0]["peer"] == b and back[0]["ext"] == x["ext"]


# ---- the exchange on numpy arrays ---------------------------------------------------------------
NQ = 8  # state fields per slot


def padded_reference(cfg, glob):
    """The undivided grid's padded arrays (slots -G..N+G per active axis):
    the periodic wrap of the interior on periodic axes, NaN beyond outflow
    boundaries (filled there by the outflow pass, not by the exchange) except
    the slot N of an outflow axis, which holds the upper boundary face (glob
    has N + 1 slots per active axis, like a face array)."""
    G, nd = G_of(cfg), cfg["ndim"]
    N = dims(cfg)
    idx, top = [], []
    for d in range(3):
        if d >= nd:
            idx.append(np.zeros(1, dtype=int))
            top.append(0)
        else:
            i = np.arange(-G, N[d] + G + 1)
            per = cfg["bc"][2 * d] == "periodic"
            idx.append(np.mod(i, N[d]) if per else i)
            top.append(N[d] - 1 if per else N[d])
    ref = np.full((NQ, len(idx[2]), len(idx[1]), len(idx[0])), np.nan)
    for q in range(NQ):
        for kk, k in enumerate(idx[2]):
            for jj, j in enumerate(idx[1]):
                for ii, i in enumerate(idx[0]):
                    if 0 <= i <= top[0] and 0 <= j <= top[1] and 0 <= k <= top[2]:
                        ref[q, kk, jj, ii] = glob[q, k, j, i]
    return ref


def glob_shape(cfg):
    N = dims(cfg)
    return (NQ,) + tuple(N[d] + (1 if d < cfg["ndim"] else 0) for d in (2, 1, 0))


def brick_arrays(cfg, parts, b, glob, rng):
    """A brick's padded arrays: its interior from the whole grid (with the
    upper boundary slot of an outflow axis on the last brick), noise in the
    ghosts."""
    G, nd = G_of(cfg), cfg["ndim"]
    lo, n = mhd.domain_brick(cfg, parts, b)
    N = dims(cfg)
    g = [G if d < nd else 0 for d in range(3)]
    ext = [n[d] + 2 * g[d] + (1 if d < nd else 0) for d in range(3)]
    e = [n[d] + (1 if d < nd and cfg["bc"][2 * d] != "periodic" and lo[d] + n[d] == N[d] else 0)
         for d in range(3)]
    a = rng.normal(size=(NQ, ext[2], ext[1], ext[0])) + 1e3
    a[:, g[2]:g[2] + e[2], g[1]:g[1] + e[1], g[0]:g[0] + e[0]] = \
        glob[:, lo[2]:lo[2] + e[2], lo[1]:lo[1] + e[1], lo[0]:lo[0] + e[0]]
    return a, g


def box_view(a, g, x):
    s = tuple(slice(x["lo"][d] + g[d], x["lo"][d] + g[d] + x["ext"][d]) for d in (2, 1, 0))
    return (slice(None),) + s


def pack(a, g, boxes):
    """Field-major per box, slots x fastest: the buffer layout of mhd_halo_box."""
    total = sum(int(np.prod(x["ext"])) for x in boxes)
    buf = np.empty(NQ * total)
    for x in boxes:
        c = int(np.prod(x["ext"]))
        buf[NQ * x["offset"]:NQ * (x["offset"] + c)] = a[box_view(a, g, x)].reshape(NQ, c).ravel()
    return buf


def unpack(a, g, boxes, buf):
    for x in boxes:
        c = int(np.prod(x["ext"]))
        shape = (NQ,) + tuple(x["ext"][d] for d in (2, 1, 0))
        a[box_view(a, g, x)] = buf[NQ * x["offset"]:NQ * (x["offset"] + c)].reshape(shape)


def deliver(send_boxes, src_buf, recv_boxes, dst_buf, src_brick):
    """Copy each box b sends in direction o into the receiver's box from -o."""
    for x in send_boxes:
        r = [y for y in recv_boxes[x["peer"]] if y["dir"] == tuple(-o for o in x["dir"])][0]
        c = NQ * int(np.prod(x["ext"]))
        dst_buf[x["peer"]][NQ * r["offset"]:NQ * r["offset"] + c] = src_buf[NQ * x["offset"]:NQ * x["offset"] + c]


def check_brick(cfg, parts, b, a, g, ref, recv_boxes):
    """Every slot the exchange filled equals the undivided grid's value."""
    lo, n = mhd.domain_brick(cfg, parts, b)
    G = G_of(cfg)
    for x in recv_boxes:
        got = a[box_view(a, g, x)]
        sl = tuple(slice(x["lo"][d] + lo[d] + g[d], x["lo"][d] + lo[d] + g[d] + x["ext"][d]) for d in (2, 1, 0))
        want = ref[(slice(None),) + sl]
        assert not np.isnan(want).any()
        np.testing.assert_array_equal(got, want)
    # and the interior is untouched
    inner = (slice(None),) + tuple(slice(g[d], g[d] + n[d]) for d in (2, 1, 0))
    sl = (slice(None),) + tuple(slice(lo[d] + g[d], lo[d] + g[d] + n[d]) for d in (2, 1, 0))
    np.testing.assert_array_equal(a[inner], ref[sl])
    assert G >= 2


@pytest.mark.parametrize("name,cfg,parts", CASES, ids=[c[0] for c in CASES])
def test_exchange_fills_ghosts_with_the_undivided_grid(name, cfg, parts):
    rng = np.random.default_rng(11)
    glob = rng.normal(size=glob_shape(cfg))
    ref = padded_reference(cfg, glob)
    nb = nbricks(parts)
    arrs = [brick_arrays(cfg, parts, b, glob, rng) for b in range(nb)]
    send = [mhd.domain_halo(cfg, parts, b, True) for b in range(nb)]
    recv = [mhd.domain_halo(cfg, parts, b, False) for b in range(nb)]
    bufs = [pack(a, g, send[b]) for b, (a, g) in enumerate(arrs)]
    rbufs = [np.full(NQ * sum(int(np.prod(x["ext"])) for x in recv[b]), np.nan) for b in range(nb)]
    for b in range(nb):
        deliver(send[b], bufs[b], recv, rbufs, b)
    for b, (a, g) in enumerate(arrs):
        assert not np.isnan(rbufs[b]).any()       # every receive slot was delivered
        unpack(a, g, recv[b], rbufs[b])
        check_brick(cfg, parts, b, a, g, ref, recv[b])


# ---- two gloo ranks, one brick each ---------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_worker(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2511_20337_b300 import workloads as W2
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = W2.base_cfg(*case[0], **case[1])
        parts = case[2]
        rng = np.random.default_rng(5)        # every rank draws the same whole grid
        glob = rng.normal(size=glob_shape(cfg))
        ref = padded_reference(cfg, glob)
        a, g = brick_arrays(cfg, parts, rank, glob, np.random.default_rng(100 + rank))
        send = mhd.domain_halo(cfg, parts, rank, True)
        recv_all = {b: mhd.domain_halo(cfg, parts, b, False) for b in range(world)}
        buf = pack(a, g, send)
        rbuf = np.full(NQ * sum(int(np.prod(x["ext"])) for x in recv_all[rank]), np.nan)
        reqs, inbox = [], []
        # post the receives, then the sends (non-blocking), as the paper's exchange does
        for x in recv_all[rank]:
            c = NQ * int(np.prod(x["ext"]))
            if x["peer"] == rank:
                continue
            t = torch.empty(c, dtype=torch.float64)
            tag = 1 + (x["dir"][0] + 1) + 3 * (x["dir"][1] + 1) + 9 * (x["dir"][2] + 1)
            reqs.append(dist.irecv(t, src=x["peer"], tag=tag))
            inbox.append((x, t))
        for x in send:
            c = NQ * int(np.prod(x["ext"]))
            chunk = buf[NQ * x["offset"]:NQ * x["offset"] + c]
            back = tuple(-o for o in x["dir"])
            if x["peer"] == rank:                 # a periodic axis with one brick: to itself
                r = [y for y in recv_all[rank] if y["dir"] == back][0]
                rbuf[NQ * r["offset"]:NQ * r["offset"] + c] = chunk
                continue
            tag = 1 + (back[0] + 1) + 3 * (back[1] + 1) + 9 * (back[2] + 1)   # the receiver's direction
            reqs.append(dist.isend(torch.from_numpy(chunk.copy()), dst=x["peer"], tag=tag))
        for r_ in reqs:
            r_.wait()
        for x, t in inbox:
            c = NQ * int(np.prod(x["ext"]))
            rbuf[NQ * x["offset"]:NQ * x["offset"] + c] = t.numpy()
        assert not np.isnan(rbuf).any()
        unpack(a, g, recv_all[rank], rbuf)
        check_brick(cfg, parts, rank, a, g, ref, recv_all[rank])
        q.put((rank, "ok"))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [
    ((3, (9, 6, 5), (0, 0, 0), (1, 1, 1)), {"recon": "wenoz"}, (2, 1, 1)),
    ((2, (8, 9), (0, 0), (1, 1)), {"bc": ["periodic", "periodic", "outflow", "outflow", "periodic", "periodic"]}, (1, 2)),
], ids=["3d-periodic-x-split", "2d-outflow-y-split"])
def test_two_gloo_ranks_exchange_their_bricks_halos(case):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, case, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, msg = q.get(timeout=180)
            out[rank] = msg
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert out == {0: "ok", 1: "ok"}
