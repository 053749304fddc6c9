"""One periodic box over several ranks: the strict slab segmentation of the
paper (Sec. 2.1), each rank owning the particles of its own x range.

The exchange protocol (host logic; every rank's compute runs in the GPU
library through cso_density / cso_fof / cso_levels):

  1. ghosts: each rank sends the particles within W = max(b, l_FoF) of its two
     x edges to the neighbouring ranks (W rounded up to a grid unit);
  2. kernel sums of the rank's own particles, its ghosts counting as
     neighbours (exact: every neighbour within b is own or ghost);
  3. the sums of the particles a rank sent as ghosts go back to the ranks that
     hold them, so every ghost's density is exact too;
  4. L0 groups over own + ghost particles; a link across a slab edge joins a
     local group to a ghost, and the ghost's owner knows that ghost's own
     local group: each rank reports (its label of the ghost, the ghost id) to
     the owner, the owners publish the label pairs, and every rank merges them
     in the same union-find (labels are particle ids; a merged group keeps the
     smallest, which is the smallest id of the group, as on one GPU);
  5. every group is processed by the rank owning its smallest-id particle:
     the other ranks send it their members (position, id, kernel sum, label);
  6. L1 and L2 on the owner, which returns the labels of the migrated
     members to their ranks and keeps the catalogue rows of its groups.

Requirements: every slab is at least 2 W wide (a particle is a ghost across one
edge at most).
The protocol is written as a generator per rank that yields its outgoing
messages ({destination rank: [message, ...]}) and receives its incoming ones
({source rank: [message, ...]}); run_distributed drives one rank over
torch.distributed (all_gather_object moves the messages; a production run
would use point-to-point sends), run_serial drives all ranks in one process.
"""
import math

import numpy as np

BOX = 1 << 21
NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


def ghost_width(params):
    """W = max(b, l_FoF) in grid units, rounded up."""
    return int(math.isqrt(int(max(params.b2, params.lfof2)))) + 1


def _wrap(d):
    return np.mod(d, BOX)


def slab_rank(rank, world, pos, ids, edges, params, ops):
    """The protocol for one rank (a generator, see the module docstring).
    pos int32 [n, 3] and ids uint64 [n] are this rank's own particles (x in
    [edges[rank], edges[rank + 1])).  Returns a dict with sigma, l0, l1, l2 of
    the own particles (input order) and the catalogue rows of the groups this
    rank owns."""
    pos = np.ascontiguousarray(pos, np.int32)
    ids = np.ascontiguousarray(ids).view(np.uint64)
    n = pos.shape[0]
    lo, hi = int(edges[rank]), int(edges[rank + 1])
    W = ghost_width(params)
    if world < 2 or min(np.diff(np.asarray(edges))) < 2 * W:
        raise ValueError("slab decomposition needs at least 2 ranks and slabs at least %d grid units wide" % (2 * W))
    left, right = (rank - 1) % world, (rank + 1) % world
    x = pos[:, 0].astype(np.int64)
    near_lo = np.nonzero(_wrap(x - lo) < W)[0]
    near_hi = np.nonzero(_wrap(hi - 1 - x) < W)[0]

    def to_neighbours(msg_lo, msg_hi):
        # with two ranks both neighbours are the same rank: both messages go there
        out = {}
        out.setdefault(left, []).append(msg_lo)
        out.setdefault(right, []).append(msg_hi)
        return out

    # 1. ghosts to the neighbours ("L": from my low edge, "R": from my high edge)
    inbox = yield to_neighbours(("ghost", "L", pos[near_lo], ids[near_lo]), ("ghost", "R", pos[near_hi], ids[near_hi]))
    ghosts = []  # (source, tag, pos, ids)
    for src, msgs in inbox.items():
        for m in msgs:
            if m[0] == "ghost":
                ghosts.append((src, m[1], m[2], m[3]))
    gpos = np.concatenate([g[2] for g in ghosts]) if ghosts else np.zeros((0, 3), np.int32)
    gids = np.concatenate([g[3] for g in ghosts]) if ghosts else np.zeros(0, np.uint64)
    ng = gpos.shape[0]

    # 2. kernel sums of the own particles; 3. the ghosts' sums come back
    allpos = np.concatenate([pos, gpos])
    allids = np.concatenate([ids, gids])
    sigma = ops.density(allpos, n)
    inbox = yield to_neighbours(("sigma", "L", sigma[near_lo]), ("sigma", "R", sigma[near_hi]))
    gsig = np.empty(ng, np.int64)
    off = 0
    for src, tag, gp, _ in ghosts:
        got = [m[2] for m in inbox.get(src, []) if m[0] == "sigma" and m[1] == tag]
        assert len(got) == 1 and got[0].size == gp.shape[0]
        gsig[off:off + gp.shape[0]] = got[0]
        off += gp.shape[0]

    # 4. L0 over own + ghosts, then the cross-edge merge
    l0loc = ops.fof(allpos, allids, np.concatenate([sigma, gsig]))
    reports = {}
    off = n
    for src, tag, gp, gi in ghosts:
        lab = l0loc[off:off + gp.shape[0]]
        m = lab != NONE
        reports.setdefault(src, []).append(("report", gi[m], lab[m]))
        off += gp.shape[0]
    inbox = yield reports
    pairs = []
    id_index = {int(v): k for k, v in enumerate(ids)} if n else {}
    for src, msgs in inbox.items():
        for m in msgs:
            if m[0] != "report" or m[1].size == 0:
                continue
            mine = l0loc[np.fromiter((id_index[int(v)] for v in m[1]), np.int64, m[1].size)]
            pairs.append(np.stack([mine, m[2]], axis=1))
    pairs = np.concatenate(pairs) if pairs else np.zeros((0, 2), np.uint64)
    inbox = yield {r: [("pairs", pairs)] for r in range(world)}
    parent = {}

    def find(a):
        root = a
        while parent.get(root, root) != root:
            root = parent[root]
        while parent.get(a, a) != root:
            parent[a], a = root, parent[a]
        return root

    for src in sorted(inbox):
        for m in inbox[src]:
            if m[0] != "pairs":
                continue
            for a, b in m[1].tolist():
                ra, rb = find(a), find(b)
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
    own_lab = l0loc[:n]
    dense = own_lab != NONE
    l0 = np.full(n, NONE, np.uint64)
    if dense.any():
        u, inv = np.unique(own_lab[dense], return_inverse=True)
        l0[dense] = np.array([find(int(v)) for v in u], np.uint64)[inv]

    # 5. group owners: the rank holding the group's smallest-id particle
    labs = np.unique(l0[dense])
    owned = labs[np.isin(labs, ids)]
    inbox = yield {r: [("owned", owned)] for r in range(world)}
    owner_of = {}
    for src, msgs in inbox.items():
        for m in msgs:
            if m[0] == "owned":
                for v in m[1].tolist():
                    owner_of[v] = src
    go = np.array([owner_of[int(v)] for v in l0[dense]], np.int64) if dense.any() else np.zeros(0, np.int64)
    didx = np.nonzero(dense)[0]
    out = {}
    for r in np.unique(go):
        if r == rank:
            continue
        k = didx[go == r]
        out.setdefault(int(r), []).append(("members", pos[k], ids[k], sigma[k], l0[k]))
    inbox = yield out

    # 6. L1 / L2 of the owned groups on this rank
    keep = didx[go == rank]
    mpos, mids, msig, ml0, msrc = [pos[keep]], [ids[keep]], [sigma[keep]], [l0[keep]], [np.full(keep.size, rank)]
    for src, msgs in inbox.items():
        for m in msgs:
            if m[0] == "members":
                mpos.append(m[1]); mids.append(m[2]); msig.append(m[3]); ml0.append(m[4])
                msrc.append(np.full(m[2].size, src))
    mpos, mids, msig, ml0, msrc = (np.concatenate(a) for a in (mpos, mids, msig, ml0, msrc))
    if mids.size:
        l1m, l2m, halos = ops.levels(mpos, mids, msig, ml0)
    else:
        l1m = l2m = np.zeros(0, np.uint64)
        halos = None
    back = {}
    for r in np.unique(msrc):
        if r == rank:
            continue
        m = msrc == r
        back.setdefault(int(r), []).append(("labels", mids[m], l1m[m], l2m[m]))
    inbox = yield back
    l1 = np.full(n, NONE, np.uint64)
    l2 = np.full(n, NONE, np.uint64)
    mine = msrc == rank
    l1[keep] = l1m[mine]
    l2[keep] = l2m[mine]
    for src, msgs in inbox.items():
        for m in msgs:
            if m[0] == "labels" and m[1].size:
                k = np.fromiter((id_index[int(v)] for v in m[1]), np.int64, m[1].size)
                l1[k] = m[2]
                l2[k] = m[3]
    return {"sigma": sigma, "l0": l0, "l1": l1, "l2": l2, "halos": halos,
            "ghosts": int(ng), "migrated_in": int((~mine).sum())}


def run_serial(gens):
    """Drive the ranks' generators in lockstep in one process."""
    world = len(gens)
    outs = [next(g) for g in gens]
    results = [None] * world
    live = set(range(world))
    while live:
        inboxes = [{} for _ in range(world)]
        for src in range(world):
            for dst, msgs in (outs[src] or {}).items():
                inboxes[dst].setdefault(src, []).extend(msgs)
        for r in list(live):
            try:
                outs[r] = gens[r].send(inboxes[r])
            except StopIteration as e:
                results[r] = e.value
                outs[r] = {}
                live.discard(r)
    return results


def run_distributed(gen, dist, rank, world):
    """Drive this rank's generator over torch.distributed; every exchange is one
    all_gather_object of the ranks' outgoing messages."""
    out = next(gen)
    while True:
        gathered = [None] * world
        dist.all_gather_object(gathered, out)
        inbox = {src: (g or {}).get(rank, []) for src, g in enumerate(gathered)}
        try:
            out = gen.send(inbox)
        except StopIteration as e:
            return e.value


class GpuOps:
    """The rank's compute through the GPU library (one context per rank)."""

    def __init__(self, ctx, params):
        self.ctx, self.p = ctx, params

    def density(self, pos, n_query):
        from . import cso
        return cso.cso_density(self.ctx.h, pos, n_query, self.p)

    def fof(self, pos, ids, sigma):
        from . import cso
        return cso.cso_fof(self.ctx.h, pos, ids, sigma, self.p)

    def levels(self, pos, ids, sigma, l0):
        from . import cso
        return cso.cso_levels(self.ctx.h, pos, ids, sigma, l0, self.p)
