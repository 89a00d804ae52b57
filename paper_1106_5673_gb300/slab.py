"""One-dimensional slab decomposition of the lattice along t (Sec. 5.2 of the
paper: the lattice is cut into slabs, each GPU keeps its slab plus a border
of neighbouring sites, and the border is refreshed by a transfer before
every application of the Dirac operator).

Host-side logic only: partitioning, the halo ranges, packing and unpacking
of the one-slice vector halo and the link halo (one full slice on each side,
enough for the hop and for the six staples of the gauge force), the sign of
the antiperiodic boundary, and the FP64 reduction of CG scalars.  The local
operator is passed in: on a GPU, the library's hop on the padded local
lattice (`gpu_local_hop`); any other callable with the same contract works.

Layout of a rank's padded lattice: extents (Lx, Ly, Lz, lt + 4) with lt = Lt
/ world (even, so that a site keeps its parity); slices t_pad = 0 and lt + 3
are unused padding (identity links, zero vectors), t_pad = 1 holds the halo
from the rank below (global t0 - 1), t_pad = 2 .. lt + 1 the rank's own slab
(global t0 .. t0 + lt - 1), t_pad = lt + 2 the halo from the rank above
(global t0 + lt).  With S = Lx Ly Lz sites per slice, slice t of a field on
one parity (index lex/2) is the contiguous range [t S/2, (t+1) S/2): every
halo is one contiguous block, and the rank's own part of a vector sits at
[S, S + lt S/2) of the padded one.

The antiperiodic fermion boundary is carried by the halos: a vector slice
that crosses the global boundary t = Lt-1 -> 0 (rank 0's lower halo, the last
rank's upper halo) is sent with its sign flipped; the padded lattice's own
boundary only touches padding and halo outputs, which are discarded.

Data plane on GPUs (not run here: every box of this build has one GPU): the
halo slices are copied into each GPU's own memory (peer copies or NCCL
send/recv of the packed slices) before the local hop; no GPU reads another's
memory during a kernel.
"""
import numpy as np


class SlabLayout:
    """Partition of a (Lx, Ly, Lz, Lt) lattice into `world` slabs along t."""

    def __init__(self, dims, world, rank):
        Lx, Ly, Lz, Lt = (int(d) for d in dims)
        if world < 1 or not 0 <= rank < world:
            raise ValueError("bad rank %d of %d" % (rank, world))
        if Lt % world or (Lt // world) % 2:
            raise ValueError("Lt = %d must split into %d even slabs" % (Lt, world))
        if any(d % 2 for d in (Lx, Ly, Lz)):
            raise ValueError("every extent must be even")
        self.dims, self.world, self.rank = (Lx, Ly, Lz, Lt), world, rank
        self.S = Lx * Ly * Lz                  # sites per time slice
        self.lt = Lt // world                  # slices per rank
        self.t0 = rank * self.lt               # first global slice of this rank
        self.local_dims = (Lx, Ly, Lz, self.lt)
        self.pad_dims = (Lx, Ly, Lz, self.lt + 4)
        self.Vh_loc = self.S * self.lt // 2
        self.Vh_pad = self.S * (self.lt + 4) // 2

    # ---- index maps (global lexicographic <-> this rank's local one)
    def local_to_global_lex(self, lex_local):
        return np.asarray(lex_local, np.int64) + self.t0 * self.S

    def owner_of_global_lex(self, lex):
        return (np.asarray(lex, np.int64) // self.S) // self.lt

    def global_to_local_lex(self, lex):
        lex = np.asarray(lex, np.int64)
        if np.any(self.owner_of_global_lex(lex) != self.rank):
            raise ValueError("site not on this rank")
        return lex - self.t0 * self.S

    # ---- slices of one-parity fields (index lex/2) and of links
    def vec_slice(self, t):
        """Half-index range of slice t of a one-parity field on this rank's
        local (unpadded) lattice."""
        return slice(t * self.S // 2, (t + 1) * self.S // 2)

    def take_local_vector(self, v_global):
        """This rank's part of a global one-parity field [V/2, 3]."""
        return v_global[self.t0 * self.S // 2:(self.t0 + self.lt) * self.S // 2]

    def take_local_links(self, U_global):
        """This rank's links [4, S lt, 3, 3] of a global field [4, V, 3, 3]."""
        return U_global[:, self.t0 * self.S:(self.t0 + self.lt) * self.S]

    def boundary_vectors(self, v_local):
        """The slices a rank sends: (lowest slice -> rank below, highest slice
        -> rank above)."""
        return v_local[self.vec_slice(0)], v_local[self.vec_slice(self.lt - 1)]

    def boundary_links(self, U_local):
        S = self.S
        return U_local[:, :S], U_local[:, (self.lt - 1) * S:]

    # ---- padded local lattice
    def pad_vector(self, v_local, halo_lo, halo_hi):
        S2 = self.S // 2
        out = np.zeros((self.Vh_pad,) + v_local.shape[1:], v_local.dtype)
        out[S2:2 * S2] = halo_lo
        out[2 * S2:2 * S2 + self.Vh_loc] = v_local
        out[2 * S2 + self.Vh_loc:3 * S2 + self.Vh_loc] = halo_hi
        return out

    def interior(self, v_pad):
        return v_pad[self.S:self.S + self.Vh_loc]

    def pad_links(self, U_local, halo_lo, halo_hi):
        S = self.S
        out = np.zeros((4, 2 * self.Vh_pad, 3, 3), U_local.dtype)
        out[...] = np.eye(3)
        out[:, S:2 * S] = halo_lo
        out[:, 2 * S:2 * S + self.S * self.lt] = U_local
        out[:, 2 * S + self.S * self.lt:3 * S + self.S * self.lt] = halo_hi
        return out

    def vector_halo_signs(self):
        """Signs of the received (lower, upper) vector halos: -1 where the
        halo crosses the antiperiodic boundary between global slices Lt-1
        and 0."""
        return (-1.0 if self.rank == 0 else 1.0), (-1.0 if self.rank == self.world - 1 else 1.0)


class TorchComm:
    """Halo exchange and scalar reduction over torch.distributed (gloo on CPU
    tensors; on GPUs the same calls with NCCL move device buffers)."""

    def __init__(self, dist):
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    def exchange(self, to_lo, to_hi):
        """Sends to_lo to the rank below and to_hi to the rank above (periodic
        in t); returns (from the rank below, from the rank above)."""
        import torch
        if self.world == 1:
            return to_hi.copy(), to_lo.copy()
        lo, hi = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        a, b = torch.from_numpy(np.ascontiguousarray(to_lo)), torch.from_numpy(np.ascontiguousarray(to_hi))
        r_lo, r_hi = torch.empty_like(b), torch.empty_like(a)
        # tags tell the two slices apart when the rank below and the rank
        # above are the same rank (two ranks): tag 1 carries a rank's highest
        # slice (the receiver's lower halo), tag 0 its lowest (the upper halo)
        ops = [self.dist.P2POp(self.dist.isend, a, lo, tag=0), self.dist.P2POp(self.dist.irecv, r_lo, lo, tag=1),
               self.dist.P2POp(self.dist.isend, b, hi, tag=1), self.dist.P2POp(self.dist.irecv, r_hi, hi, tag=0)]
        for req in self.dist.batch_isend_irecv(ops):
            req.wait()
        return r_lo.numpy(), r_hi.numpy()

    def allreduce(self, x):
        """FP64 sum over ranks of a float."""
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64)
        self.dist.all_reduce(t)
        return float(t.item())


class ThreadComm:
    """The same exchange between ranks that run as threads of one process
    (one slab per thread; a barrier orders the hand-over).  For checking the
    decomposition's data plane on a single device."""

    def __init__(self, shared, rank, world):
        self.s, self.rank, self.world = shared, rank, world

    @staticmethod
    def shared(world):
        import threading
        return {"barrier": threading.Barrier(world), "box": {}}

    def exchange(self, to_lo, to_hi):
        box, bar = self.s["box"], self.s["barrier"]
        box[self.rank] = (np.array(to_lo), np.array(to_hi))
        bar.wait()
        lo, hi = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        out = box[lo][1].copy(), box[hi][0].copy()
        bar.wait()
        return out

    def allreduce(self, x):
        box, bar = self.s["box"], self.s["barrier"]
        box[self.rank] = float(x)
        bar.wait()
        tot = sum(box[r] for r in range(self.world))
        bar.wait()
        return tot


class SlabOperator:
    """D_eo, D_oe, M_ee = m^2 - D_eo D_oe and CG over the slab decomposition.
    local_hop(pad_dims, U_pad, out_parity, v_pad) -> D restricted to
    out_parity on the padded lattice (complex [Vh_pad, 3])."""

    def __init__(self, layout, comm, local_hop, U_local):
        self.L, self.comm, self.hop = layout, comm, local_hop
        lo, hi = layout.boundary_links(U_local)
        # the rank below sends its highest slice (it becomes our lower halo)
        h_lo, h_hi = comm.exchange(lo, hi)
        self.U_pad = layout.pad_links(U_local, h_lo, h_hi)
        self.link_halos = (h_lo, h_hi)

    def halo(self, v_local):
        lo, hi = self.L.boundary_vectors(v_local)
        h_lo, h_hi = self.comm.exchange(lo, hi)
        s_lo, s_hi = self.L.vector_halo_signs()
        return s_lo * h_lo, s_hi * h_hi

    def dslash(self, out_parity, v_local):
        h_lo, h_hi = self.halo(v_local)
        out = self.hop(self.L.pad_dims, self.U_pad, out_parity, self.L.pad_vector(v_local, h_lo, h_hi))
        return np.array(self.L.interior(out))

    def apply_M(self, mass, v_local):
        return mass * mass * v_local - self.dslash(0, self.dslash(1, v_local))

    def dot(self, a, b):
        """Re <a, b> summed over ranks in FP64."""
        return self.comm.allreduce(np.vdot(a.reshape(-1), b.reshape(-1)).real)

    def cg(self, mass, shift, b, tol=1e-10, maxit=1000):
        """Plain CG for (M_ee + shift) x = b from x = 0 (the per-shift solver
        of Sec. 4.3), every scalar reduced over the ranks."""
        x = np.zeros_like(b)
        r = b.copy()
        p = b.copy()
        bb = self.dot(b, b)
        rr = bb
        it = 0
        while it < maxit and rr > tol * tol * bb:
            w = self.apply_M(mass, p) + shift * p
            alpha = rr / self.dot(p, w)
            x += alpha * p
            r -= alpha * w
            rr_new = self.dot(r, r)
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
        return x, it


def gpu_local_hop(stag, torch):
    """The library's FP64 hop on a rank's padded lattice (one context per
    padded shape, links loaded when they change)."""
    cache = {}

    def hop(pad_dims, U_pad, out_parity, v_pad):
        key = tuple(pad_dims)
        if key not in cache:
            cache[key] = [stag.Lattice(pad_dims), None]
        L, U_seen = cache[key]
        if U_seen is not U_pad:
            L.load_gauge(np.ascontiguousarray(U_pad))
            cache[key][1] = U_pad
        x = torch.from_numpy(np.ascontiguousarray(v_pad)).cuda()
        y = L.vector()
        (L.apply_deo if out_parity == 0 else L.apply_doe)(x, y)
        torch.cuda.synchronize()
        return y.cpu().numpy()

    return hop
