"""Domain decomposition of one periodic system over ranks (the distributed-
memory outlook of the paper's conclusion), host side.

Rank r owns the contiguous slab of cell layers [z0_r, z1_r) along z of the
system's linked-cell grid (at least two layers per rank, so that a rank's two
halo layers are distinct) and the molecules in it.  One force evaluation:

1. halo exchange: every rank sends the molecules of its lowest layer to the
   rank below (periodic ring) and those of its highest layer to the rank
   above; its local system is its own molecules plus the one halo layer
   received from each side, in the global box (so the library bins them as a
   single-domain run would);
2. the library evaluates the local system with its owned layers restricted
   to the slab (``atm_set_owned_layers``): 3C01 and LJ give the complete
   force of every owned molecule; the Newton-3 traversals 3C18 / 3C08 / 3C08A
   give the owned units' share, including forces on the halo layer above
   (their units reach one layer up);
3. force return: every rank sends the forces its units put on the halo layer
   above back to that layer's owner, which adds them to its molecules in the
   order it sent them;
4. energies, virials and counts are summed over the ranks.

The exchange goes through a transport: ``DistTransport`` (torch.distributed:
NCCL between GPUs, gloo on CPUs) or ``LocalRanks`` (every rank in one process,
each with its own context, messages passed in memory).  The compute goes
through a backend: ``LibraryBackend`` (the CUDA library); tests pass other
backends with the same two methods.  Cell layers always come from the
backend's own cell build, never from host arithmetic.
"""
import numpy as np

SCALARS = ("e2", "e3", "w2", "w3", "n_cand3", "n_int3", "n_cand2", "n_int2")
NEWTON3 = ("3c18", "3c08", "3c08a")


def slabs(nz, world):
    """Layer bounds [z0_r, z1_r) of the ranks: contiguous, as even as possible,
    at least two layers each (ValueError otherwise)."""
    if world < 1 or nz < 2 * world:
        raise ValueError("%d cell layers cannot give %d ranks two layers each" % (nz, world))
    q, rem = divmod(nz, world)
    sizes = [q + (1 if r < rem else 0) for r in range(world)]
    b = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
    return [(int(b[r]), int(b[r + 1])) for r in range(world)]


class RankState:
    """One rank's molecules: positions x [3, m], global ids [m] and their cell
    layers [m] (from the backend's last cell build)."""

    def __init__(self, rank, world, box, nz, x, ids, layers):
        self.rank, self.world = rank, world
        self.box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)).copy()
        self.nz = nz
        self.z0, self.z1 = slabs(nz, world)[rank]
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.ids = np.asarray(ids, dtype=np.int64)
        self.layers = np.asarray(layers, dtype=np.int64)
        if np.any((self.layers < self.z0) | (self.layers >= self.z1)):
            raise ValueError("rank %d holds molecules outside its slab" % rank)


def distribute(x, layers, box, nz, world):
    """Initial partition of a whole system (x [3, N], cell layers [N] from a
    cell build of it): the RankState of every rank."""
    out = []
    for r, (z0, z1) in enumerate(slabs(nz, world)):
        sel = np.nonzero((layers >= z0) & (layers < z1))[0]
        out.append(RankState(r, world, box, nz, x[:, sel], sel, layers[sel]))
    return out


def _pack(x, ids):
    """Message of molecules: rows (x, y, z, id)."""
    return np.ascontiguousarray(np.vstack([x, ids[None, :].astype(np.float64)]).T)


def _unpack(msg):
    msg = np.asarray(msg, dtype=np.float64).reshape(-1, 4)
    return np.ascontiguousarray(msg[:, :3].T), msg[:, 3].astype(np.int64)


# ---------------------------------------------------------------- the phases

def halo_out(st):
    """Phase 1: the molecules of the lowest layer (for the rank below) and of
    the highest layer (for the rank above)."""
    lo = np.nonzero(st.layers == st.z0)[0]
    hi = np.nonzero(st.layers == st.z1 - 1)[0]
    st._sent_down = lo
    return _pack(st.x[:, lo], st.ids[lo]), _pack(st.x[:, hi], st.ids[hi])


def local_forces(st, from_below, from_above, backend, trav, trunc, prec):
    """Phase 2: evaluate own + halo molecules with the owned layers restricted
    to the slab.  Returns the forces this rank's units put on the halo layer
    above (for its owner) as a message."""
    xb, _ = _unpack(from_below)
    xa, _ = _unpack(from_above)
    m, nb = st.x.shape[1], xb.shape[1]
    xl = np.ascontiguousarray(np.concatenate([st.x, xb, xa], axis=1))
    f, res, layers = backend.forces(st.box, xl, st.z0, st.z1, trav, trunc, prec)
    st.f = np.array(f[:, :m])
    st.res = {k: res[k] for k in SCALARS if res.get(k) is not None}
    st.layers = np.asarray(layers[:m], dtype=np.int64)
    back = f[:, m + nb:] if trav in NEWTON3 else np.zeros((3, xa.shape[1]))
    return np.ascontiguousarray(back.T)


def add_returned(st, from_below_forces):
    """Phase 3: add the forces the rank below put on this rank's lowest layer
    (rows in the order phase 1 sent them)."""
    fb = np.asarray(from_below_forces, dtype=np.float64).reshape(-1, 3)
    if fb.shape[0] != st._sent_down.size:
        raise RuntimeError("returned forces do not match the halo sent")
    if fb.shape[0]:
        st.f[:, st._sent_down] += fb.T


def migrate_out(st):
    """Molecules whose last cell build put them outside the slab leave: the
    ones below z0 (periodically) for the rank below, the rest for the rank
    above.  A step moves a molecule by less than one layer."""
    out = (st.layers < st.z0) | (st.layers >= st.z1)
    below = st.layers == (st.z0 - 1) % st.nz
    above = st.layers == st.z1 % st.nz
    if np.any(out & ~below & ~above):
        raise RuntimeError("a molecule moved more than one cell layer in a step")
    msgs = (_pack(st.x[:, below], st.ids[below]), _pack(st.x[:, above], st.ids[above]))
    keep = ~out
    st.x, st.ids, st.layers = st.x[:, keep], st.ids[keep], st.layers[keep]
    return msgs


def migrate_in(st, from_below, from_above, backend):
    for msg in (from_below, from_above):
        x, ids = _unpack(msg)
        st.x = np.ascontiguousarray(np.concatenate([st.x, x], axis=1))
        st.ids = np.concatenate([st.ids, ids])
    st.layers = np.asarray(backend.layers(st.box, st.x), dtype=np.int64)


# ---------------------------------------------------------------- transports

class DistTransport:
    """Neighbour exchange and sums over torch.distributed ranks (NCCL between
    GPUs, gloo on CPUs); messages travel as float64 tensors on `device`."""

    def __init__(self, device="cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.device = device

    def _shift(self, msg, up):
        import torch
        dist = self.dist
        dst = (self.rank + 1) % self.world if up else (self.rank - 1) % self.world
        src = (self.rank - 1) % self.world if up else (self.rank + 1) % self.world
        t = torch.as_tensor(np.ascontiguousarray(msg, dtype=np.float64)).reshape(-1).to(self.device)
        ns = torch.tensor([t.numel()], dtype=torch.int64, device=self.device)
        nr = torch.zeros(1, dtype=torch.int64, device=self.device)
        for op in dist.batch_isend_irecv([dist.P2POp(dist.isend, ns, dst),
                                          dist.P2POp(dist.irecv, nr, src)]):
            op.wait()
        r = torch.zeros(int(nr.item()), dtype=torch.float64, device=self.device)
        ops = []
        if t.numel():
            ops.append(dist.P2POp(dist.isend, t, dst))
        if r.numel():
            ops.append(dist.P2POp(dist.irecv, r, src))
        if ops:
            for op in dist.batch_isend_irecv(ops):
                op.wait()
        return r.cpu().numpy()

    def up(self, msg):
        """Send to the rank above, receive from the rank below."""
        return self._shift(msg, True)

    def down(self, msg):
        """Send to the rank below, receive from the rank above."""
        return self._shift(msg, False)

    def allreduce(self, vec):
        import torch
        t = torch.as_tensor(np.asarray(vec, dtype=np.float64)).to(self.device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()


def _sum_scalars(results):
    out = {}
    for k in SCALARS:
        vals = [r[k] for r in results if k in r]
        if vals:
            out[k] = int(sum(vals)) if k.startswith("n_") else float(sum(vals))
    return out


def evaluate_dist(st, backend, transport, trav="3c08", trunc="pair", prec="fp64"):
    """One force evaluation on this rank (every rank calls it): st.f receives
    the complete forces of the rank's molecules; returns the global scalars."""
    if transport.world == 1:
        f, res, layers = backend.forces(st.box, st.x, st.z0, st.z1, trav, trunc, prec)
        st.f, st.layers = np.array(f), np.asarray(layers, dtype=np.int64)
        return _sum_scalars([res])
    to_below, to_above = halo_out(st)
    from_below = transport.up(to_above)     # the rank below's highest layer
    from_above = transport.down(to_below)   # the rank above's lowest layer
    back = local_forces(st, from_below, from_above, backend, trav, trunc, prec)
    add_returned(st, transport.up(back))
    keys = [k for k in SCALARS if k in st.res]
    tot = transport.allreduce([float(st.res[k]) for k in keys])
    return {k: (int(round(v)) if k.startswith("n_") else float(v)) for k, v in zip(keys, tot)}


class LocalRanks:
    """Every rank in one process (each with its own backend), the messages
    passed in memory: the same phases as evaluate_dist."""

    def __init__(self, states, backends):
        self.states, self.backends = states, backends
        self.world = len(states)

    def evaluate(self, trav="3c08", trunc="pair", prec="fp64"):
        R = self.world
        if R == 1:
            st, be = self.states[0], self.backends[0]
            f, res, layers = be.forces(st.box, st.x, st.z0, st.z1, trav, trunc, prec)
            st.f, st.layers = np.array(f), np.asarray(layers, dtype=np.int64)
            return _sum_scalars([res])
        out = [halo_out(st) for st in self.states]          # (to_below, to_above)
        backs = [local_forces(st, out[(r - 1) % R][1], out[(r + 1) % R][0], self.backends[r],
                              trav, trunc, prec) for r, st in enumerate(self.states)]
        for r, st in enumerate(self.states):
            add_returned(st, backs[(r - 1) % R])
        return _sum_scalars([st.res for st in self.states])

    def migrate(self):
        R = self.world
        msgs = [migrate_out(st) for st in self.states]      # (to_below, to_above)
        for r, st in enumerate(self.states):
            migrate_in(st, msgs[(r + 1) % R][0], msgs[(r - 1) % R][1], self.backends[r])

    def gather(self, n):
        """Forces of all ranks in global-id order [3, n]."""
        f = np.zeros((3, n))
        for st in self.states:
            f[:, st.ids] = st.f
        return f


# ---------------------------------------------------------------- the CUDA backend

class LibraryBackend:
    """Force evaluation of a local system by the CUDA library (one context,
    re-created when the local molecule count changes)."""

    def __init__(self, rc=2.5, nu=0.073, device=0, stream=None):
        from paper_2510_21230_gb300 import atm3
        self.atm3 = atm3
        self.rc, self.nu, self.device, self.stream = rc, nu, device, stream
        self.sys = None
        self.key = None

    def nz(self, box):
        return int(self.atm3.cell_grid(box, self.rc)[2])

    def _system(self, box, n):
        key = (tuple(np.broadcast_to(box, (3,))), n)
        if self.key != key:
            if self.sys is not None:
                self.sys.close()
            self.sys = self.atm3.AtmSystem(box, n, rc=self.rc, nu=self.nu, device=self.device,
                                           stream=self.stream)
            self.key = key
        return self.sys

    def layers(self, box, x):
        s = self._system(box, x.shape[1])
        s.set_owned_layers(0, self.nz(box))
        s.set_state(x)
        s.build_cells()
        c = s.get_cells()
        return c["cell_of"] // (int(c["ncell"][0]) * int(c["ncell"][1]))

    def forces(self, box, x, z0, z1, trav, trunc, prec):
        s = self._system(box, x.shape[1])
        s.set_owned_layers(z0, z1)
        s.set_state(x)
        s.build_cells()
        res = s.compute_forces(trav, trunc, prec)
        c = s.get_cells()
        layers = c["cell_of"] // (int(c["ncell"][0]) * int(c["ncell"][1]))
        return s.get_forces("total"), res, layers

    def close(self):
        if self.sys is not None:
            self.sys.close()
            self.sys = None
