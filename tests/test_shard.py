"""The FMM partitioned over several GPUs (Sec. "Numerical solution": every process owns a part
of the octree and receives its locally essential tree): the library's plan and locally
essential trees, and the exchange module, on CPU.

The tree is built here from its definition on a clustered point cloud (split while a box
holds more than 24 points), with the interaction lists written out from their definitions:
  U(B) -- leaves adjacent to the leaf B (B included);
  V(B) -- children of the colleagues of B's parent not adjacent to B;
  W(B) -- for a leaf B, descendants of its colleagues not adjacent to B whose parent is;
  X(B) -- the boxes A with B in W(A).
Checks: the plan covers every leaf once in contiguous Morton ranges of balanced cost; each
rank's locally essential tree holds exactly the boxes its lists need from other ranks; and on
two gloo ranks that each hold only their own leaves' densities, the exchanged data give every
rank the same near-field sums and upward moments as one process holding everything.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KEY_LEVEL = 10


def _morton(ijk):
    k = np.zeros(len(ijk), np.int64)
    for bit in range(KEY_LEVEL - 1, -1, -1):
        for c in range(3):
            k = (k << 1) | ((ijk[:, c] >> bit) & 1)
    return k


def build_tree(n=3000, cap=24, max_level=7, seed=11):
    rng = np.random.default_rng(seed)
    pts = np.concatenate([rng.uniform(0, 1, (n // 2, 3)), 0.5 + 0.08 * rng.normal(size=(n - n // 2, 3))])
    pts = np.clip(pts, 0, 1 - 1e-9)
    ijk = np.floor(pts * (1 << KEY_LEVEL)).astype(np.int64)
    order = np.argsort(_morton(ijk), kind="stable")
    pts = pts[order]
    keys = _morton(ijk[order])
    level, anchor, parent, rng_ = [0], [(0, 0, 0)], [-1], [(0, len(pts))]
    head = 0
    while head < len(level):
        b = head
        head += 1
        lo, hi = rng_[b]
        if hi - lo <= cap or level[b] >= max_level:
            continue
        l1 = level[b] + 1
        for o in range(8):
            a = (2 * anchor[b][0] + (o >> 2 & 1), 2 * anchor[b][1] + (o >> 1 & 1), 2 * anchor[b][2] + (o & 1))
            k0 = _morton(np.array([[a[0] << (KEY_LEVEL - l1), a[1] << (KEY_LEVEL - l1), a[2] << (KEY_LEVEL - l1)]]))[0]
            s, e = np.searchsorted(keys, [k0, k0 + (1 << (3 * (KEY_LEVEL - l1)))])
            if e > s:
                level.append(l1)
                anchor.append(a)
                parent.append(b)
                rng_.append((int(s), int(e)))
    level, anchor, parent, rng_ = (np.array(v, np.int32) for v in (level, anchor, parent, rng_))
    return pts, level, anchor, parent, rng_


def build_lists(level, anchor, parent):
    nb = len(level)
    size = (1 << (KEY_LEVEL - level)).astype(np.int64)
    lo = anchor.astype(np.int64) * size[:, None]
    hi = lo + size[:, None]
    children = [[] for _ in range(nb)]
    for b in range(1, nb):
        children[parent[b]].append(b)
    leaf = np.array([not c for c in children])

    def adjacent(a, b):
        return bool(np.all(lo[a] <= hi[b]) and np.all(lo[b] <= hi[a]))

    def desc(b):
        out, stack = [], list(children[b])
        while stack:
            d = stack.pop()
            out.append(d)
            stack.extend(children[d])
        return out

    colleagues = [[c for c in range(nb) if level[c] == level[b] and adjacent(b, c)] for b in range(nb)]
    U, V, W = ([[] for _ in range(nb)] for _ in range(3))
    for b in range(nb):
        if b > 0:
            V[b] = sorted(ch for c in colleagues[parent[b]] for ch in children[c] if not adjacent(ch, b))
        if leaf[b]:
            U[b] = sorted(c for c in range(nb) if leaf[c] and adjacent(b, c))
            W[b] = sorted(d for c in colleagues[b] if c != b for d in desc(c)
                          if not adjacent(d, b) and adjacent(parent[d], b))
    X = [[] for _ in range(nb)]
    for a in range(nb):
        for b in W[a]:
            X[b].append(a)

    def csr(lists):
        off = np.zeros(nb + 1, np.int32)
        off[1:] = np.cumsum([len(v) for v in lists])
        idx = np.array([i for v in lists for i in v], np.int32)
        return off, idx

    return {"U": csr(U), "V": csr(V), "W": csr(W), "X": csr(X)}, leaf, (U, V, W, X)


@pytest.fixture(scope="module")
def tree():
    import paper_1612_04082_gb300 as K
    pts, level, anchor, parent, rng_ = build_tree()
    lists, leaf, raw = build_lists(level, anchor, parent)
    tv = K.TreeView({"level": level, "anchor": anchor, "parent": parent, "src": rng_, "trg": rng_}, lists)
    return K, tv, pts, leaf, raw, rng_, parent


def _ancestors(b, parent):
    out = []
    while b >= 0:
        out.append(b)
        b = parent[b]
    return out


@pytest.mark.parametrize("n_ranks", [1, 2, 3, 5])
def test_plan_and_locally_essential_trees(tree, n_ranks):
    K, tv, pts, leaf, (U, V, W, X), rng_, parent = tree
    owner, order, rank_cost = K.kfmm_shard_plan(tv, n_ranks)
    leaves = np.flatnonzero(leaf)
    assert sorted(order) == sorted(leaves)                      # every leaf once
    assert np.all(np.diff(rng_[order, 0]) > 0)                  # Morton order = sorted order
    seq = owner[order]
    assert np.all(np.diff(seq) >= 0) and set(seq) == set(range(n_ranks))  # contiguous ranges
    cost = {b: (rng_[b, 1] - rng_[b, 0]) * sum(rng_[s, 1] - rng_[s, 0] for s in U[b]) + 2 * (rng_[b, 1] - rng_[b, 0])
            + 1 for b in leaves}
    assert np.isclose(rank_cost.sum(), sum(cost.values()))
    assert rank_cost.max() <= rank_cost.sum() / n_ranks + max(cost.values()) + 1e-9
    for b in range(len(owner)):                                 # box owners from their leaves
        below = {owner[d] for d in leaves if b in _ancestors(d, parent)}
        assert owner[b] == (below.pop() if len(below) == 1 else -1)
    for r in range(n_ranks):
        src, up, shared = K.kfmm_shard_let(tv, owner, r)
        mine = [b for b in leaves if owner[b] == r]
        side = sorted({a for b in mine for a in _ancestors(b, parent)})
        need_src = {s for b in mine for s in U[b]} | {s for b in side for s in X[b]}
        need_up = {s for b in side for s in V[b]} | {s for b in mine for s in W[b]}
        assert set(src) == {s for s in need_src if owner[s] != r}
        assert all(leaf[s] for s in src)
        assert set(up) == {s for s in need_up if owner[s] not in (r, -1)}
        assert set(shared) == {s for s in need_up if owner[s] == -1} | {b for b in side if owner[b] == -1}
        if n_ranks == 1:
            assert len(src) == len(up) == len(shared) == 0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "1"  # many tiny oracle sums: no thread start-up per call
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle as O
        import paper_1612_04082_gb300 as K
        from paper_1612_04082_gb300.shard import ShardExchange
        pts, level, anchor, parent, rng_ = build_tree()
        lists, leaf, (U, V, W, X) = build_lists(level, anchor, parent)
        tv = K.TreeView({"level": level, "anchor": anchor, "parent": parent, "src": rng_, "trg": rng_}, lists)
        ex = ShardExchange(tv, rank, world)
        dens = np.random.default_rng(5).normal(size=(len(pts), 3))
        nb = len(level)
        mine = ex.owned_leaves()
        local = np.full_like(dens, np.nan)  # this rank holds only its own leaves' densities
        for b in mine:
            local[rng_[b, 0]:rng_[b, 1]] = dens[rng_[b, 0]:rng_[b, 1]]
        have = ex.gather_sources(local)
        # near field of the rank's targets from the U lists, with the data it now holds
        near_ok = True
        for b in mine:
            t = pts[rng_[b, 0]:rng_[b, 1]]
            got = sum(O.direct_disp(t, pts[rng_[s, 0]:rng_[s, 1]], None, have[rng_[s, 0]:rng_[s, 1]]) for s in U[b])
            ref = sum(O.direct_disp(t, pts[rng_[s, 0]:rng_[s, 1]], None, dens[rng_[s, 0]:rng_[s, 1]]) for s in U[b])
            near_ok = near_ok and np.array_equal(got, ref)
        # upward moments (sums of the densities below a box): own boxes locally, shared boxes
        # by the all-reduce of partial sums, ghost boxes from their owners
        part = np.zeros((nb, 3))
        for b in range(nb):
            rows = local[rng_[b, 0]:rng_[b, 1]]
            part[b] = np.nansum(rows, axis=0)
        full = ex.gather_up(ex.reduce_shared(part))
        ref_m = np.array([dens[rng_[b, 0]:rng_[b, 1]].sum(0) for b in range(nb)])
        src, up, shared = ex.lets[rank]
        side = sorted({a for b in mine for a in _ancestors(b, parent)})
        need_up = sorted({s for b in side for s in V[b]} | {s for b in mine for s in W[b]} | set(side))
        up_ok = bool(np.allclose(full[need_up], ref_m[need_up], rtol=1e-12, atol=1e-12))
        q.put((rank, near_ok, up_ok, len(src), len(up), len(shared)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_exchange_their_locally_essential_trees():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, near_ok, up_ok, ns, nu, nh in res:
        assert near_ok and up_ok, (rank, near_ok, up_ok)
        assert ns > 0 and nh > 0  # the ranks did exchange sources and share coarse boxes
