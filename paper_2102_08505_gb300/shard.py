"""Host-side logic for runs on several GPUs of one node (one process per GPU).

Three ways to use several GPUs:
  - replicas: each rank purifies its own Hamiltonian, no collective on the data path;
  - batched SP2: whole matrices are dealt to ranks (deal), only statistics are gathered;
  - the row-block split of one SP2 run (row_block_sp2): rank r owns a contiguous block of
    rows of X (Morton order keeps a block spatially compact).  Each iteration, a block's
    product rows need the rows of X its entries name: its own and a halo owned by other
    ranks, fetched by point-to-point exchange; the traces are the blocks' shares summed
    in rank order.  The paper places row blocks on NUMA domains (Section "Micro-Kernel
    Performance Evaluation - NUMA Aware Data"); here a block lives on one GPU.
The timed regions use a barrier and the maximum over ranks of the elapsed time.
"""
import os
import threading

import numpy as np


def rank_info():
    """(rank, local_rank, world_size) from the launcher's environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def deal(work, world):
    """Longest-processing-time assignment of items with the given work estimates to
    `world` ranks: items in decreasing work (ties by index) go to the least-loaded rank
    (ties by rank).  Deterministic, so every rank computes the same split.  Returns a
    list of sorted index lists, one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(work[i])
    return [sorted(p) for p in parts]


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks of the default process group (the value itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    """Sum of a float over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()



# ------------------------------------------------------------------ row-block split
def block_bounds(n, world):
    """Contiguous row blocks: rank r owns rows bounds[r] .. bounds[r + 1] - 1."""
    if world < 1 or n < world:
        raise ValueError("need 1 <= world <= n")
    return [(n * r) // world for r in range(world + 1)]


def owners(rows, bounds):
    """Rank owning each global row."""
    return np.searchsorted(np.asarray(bounds), np.asarray(rows), side="right") - 1


def halo_requests(idx, nnz, r0, r1, bounds):
    """Rows outside [r0, r1) that the block's stored entries name, grouped by owner:
    {rank: sorted int64 array}.  idx, nnz: numpy arrays of the block's rows."""
    live = np.arange(idx.shape[1])[None, :] < np.minimum(nnz, idx.shape[1])[:, None]
    ks = np.unique(idx[live].astype(np.int64))
    ks = ks[(ks < r0) | (ks >= r1)]
    own = owners(ks, bounds)
    return {int(q): ks[own == q] for q in np.unique(own)}


class DistComm:
    """Point-to-point exchanges and ordered sums over the default torch.distributed group
    (gloo on CPU tensors, NCCL on CUDA tensors)."""

    def __init__(self, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.device = device

    def exchange(self, sends, recvs):
        """sends[q] / recvs[q]: lists of tensors to send to / receive from rank q (shapes
        agreed beforehand; empty tensors are skipped on both sides)."""
        ops = []
        for q, ts in recvs.items():
            ops += [self.dist.P2POp(self.dist.irecv, t, q) for t in ts if t.numel()]
        for q, ts in sends.items():
            ops += [self.dist.P2POp(self.dist.isend, t.contiguous(), q) for t in ts if t.numel()]
        if ops:
            for w in self.dist.batch_isend_irecv(ops):
                w.wait()

    def reduce_scalar(self, value, op):
        import torch
        t = torch.tensor([float(value)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op={"min": self.dist.ReduceOp.MIN, "max": self.dist.ReduceOp.MAX}[op])
        return float(t.item())

    def ordered_sums(self, parts):
        """parts: k arrays of this rank's values.  Returns the k sums over all ranks, taken
        rank after rank, each rank adding its values in order to the running sums it
        receives: the sums one process adding every value in row order would get.  The
        same on every rank."""
        import torch
        parts = [np.atleast_1d(np.asarray(p, np.float64)) for p in parts]
        k = len(parts)
        run = torch.zeros(k, dtype=torch.float64, device=self.device)
        if self.rank > 0:
            self.dist.recv(run, self.rank - 1)
        acc = run.cpu().numpy().copy()
        for c in range(k):
            for v in parts[c]:
                acc[c] = acc[c] + v
        out = torch.tensor(acc, dtype=torch.float64, device=self.device)
        if self.rank + 1 < self.world:
            self.dist.send(out, self.rank + 1)
        self.dist.broadcast(out, self.world - 1)
        return out.cpu().numpy()


class LocalComm:
    """The same interface for ranks run as threads of one process (each thread a rank,
    messages handed over in memory): the row-block split exercised on one GPU, where the
    ranks' kernels never wait on one another (every exchange passes through the host)."""

    class Hub:
        def __init__(self, world):
            self.world = world
            self.cv = threading.Condition()
            self.box = {}

        def put(self, key, val):
            with self.cv:
                self.box[key] = val
                self.cv.notify_all()

        def get(self, key, timeout=120.0):
            with self.cv:
                if not self.cv.wait_for(lambda: key in self.box, timeout=timeout):
                    raise TimeoutError("rank message %r never arrived" % (key,))
                return self.box.pop(key)

    def __init__(self, hub, rank, device=None):
        self.hub, self.rank, self.world, self.device = hub, rank, hub.world, device
        self.seq = 0

    def _tag(self):
        self.seq += 1
        return self.seq

    def exchange(self, sends, recvs):
        tag = self._tag()
        for q, ts in sends.items():
            self.hub.put(("x", tag, self.rank, q), [t.clone() for t in ts])
        for q, ts in recvs.items():
            got = self.hub.get(("x", tag, q, self.rank))
            for t, g in zip(ts, got):
                if t.numel():
                    t.copy_(g)

    def reduce_scalar(self, value, op):
        tag = self._tag()
        for q in range(self.world):
            self.hub.put(("r", tag, self.rank, q), float(value))
        vals = [self.hub.get(("r", tag, q, self.rank)) for q in range(self.world)]
        return min(vals) if op == "min" else max(vals)

    def ordered_sums(self, parts):
        tag = self._tag()
        parts = [np.atleast_1d(np.asarray(p, np.float64)) for p in parts]
        acc = np.zeros(len(parts))
        if self.rank > 0:
            acc = self.hub.get(("s", tag, self.rank - 1, self.rank))
        acc = acc.copy()
        for c in range(len(parts)):
            for v in parts[c]:
                acc[c] = acc[c] + v
        if self.rank + 1 < self.world:
            self.hub.put(("s", tag, self.rank, self.rank + 1), acc)
            return self.hub.get(("t", tag, self.world - 1, self.rank))
        for q in range(self.world - 1):
            self.hub.put(("t", tag, self.rank, q), acc)
        return acc


def fetch_halo(comm, bounds, r0, idx, val, nnz, req):
    """Point-to-point halo exchange.  idx/val/nnz: torch tensors of this rank's rows (all
    ranks use the same width); req: halo_requests of this rank.  Returns (rows, idx, val,
    nnz) of the received halo rows (torch tensors on the tensors' device)."""
    import torch
    dev, w = idx.device, idx.shape[1]
    world, me = comm.world, comm.rank
    peers = [q for q in range(world) if q != me]
    empty = torch.zeros(0, dtype=torch.int64, device=dev)
    want = {q: torch.as_tensor(req[q], device=dev).to(torch.int64) if q in req else empty for q in peers}
    # 1. how many rows each peer wants from this rank
    cnt_out = {q: torch.tensor([want[q].numel()], dtype=torch.int64, device=dev) for q in peers}
    cnt_in = {q: torch.zeros(1, dtype=torch.int64, device=dev) for q in peers}
    comm.exchange({q: [cnt_out[q]] for q in peers}, {q: [cnt_in[q]] for q in peers})
    # 2. the row lists
    asked = {q: torch.zeros(int(cnt_in[q].item()), dtype=torch.int64, device=dev) for q in peers}
    comm.exchange({q: [want[q]] for q in peers}, {q: [asked[q]] for q in peers})
    # 3. the rows themselves
    sends = {}
    for q in peers:
        loc = asked[q] - r0
        sends[q] = [nnz[loc].contiguous(), idx[loc].contiguous(), val[loc].contiguous()]
    recvs = {q: [torch.zeros(want[q].numel(), dtype=nnz.dtype, device=dev),
                 torch.zeros((want[q].numel(), w), dtype=idx.dtype, device=dev),
                 torch.zeros((want[q].numel(), w), dtype=val.dtype, device=dev)] for q in peers}
    comm.exchange(sends, recvs)
    if not peers:
        z = torch.zeros(0, dtype=torch.int64, device=dev)
        return z, idx[:0], val[:0], nnz[:0]
    rows = torch.cat([want[q] for q in peers])
    return (rows, torch.cat([recvs[q][1] for q in peers]), torch.cat([recvs[q][2] for q in peers]),
            torch.cat([recvs[q][0] for q in peers]))


def row_block_sp2(comm, bounds, H_blk, nocc, tol, tau, backend, max_iter=100, stall_arm=0.1, stall_ratio=1.0):
    """One SP2 purification with the rows of X split into blocks over ranks (SPMD: every
    rank calls this with its own block).  H_blk: this rank's rows of H (the backend's
    matrix type); backend: the per-block operations (GPUBlockOps for the CUDA library).
    Per iteration: halo exchange, the block's traces summed over ranks in rank order, the
    stop rules and branch of sp2_purify, the block's product with the fused update.
    Returns (this rank's rows of D, statistics dict)."""
    r0, r1 = bounds[comm.rank], bounds[comm.rank + 1]
    n = bounds[-1]
    lo, hi = backend.bounds(H_blk, r0)
    lo, hi = comm.reduce_scalar(lo, "min"), comm.reduce_scalar(hi, "max")
    X = backend.x0(H_blk, r0, lo, hi, tau)
    st = {"iterations": 0, "branch": [], "trX": [], "trX2": [], "err": [], "emin": lo, "emax": hi,
          "halo_rows": []}
    armed = False
    it = 0
    status = "max_iter"
    while True:
        w = int(comm.reduce_scalar(backend.width(X), "max"))
        X = backend.widen(X, w)
        idx, val, nnz = backend.arrays(X)
        req = backend.halo_requests(X, r0, r1, bounds)
        halo = fetch_halo(comm, bounds, r0, idx, val, nnz, req)
        st["halo_rows"].append(int(halo[0].numel()))
        B = backend.extended(X, r0, n, halo)
        parts = backend.trace_parts(X, r0, B)
        trX, trX2 = comm.ordered_sums(parts)
        err = abs(trX - trX2) / n
        st["trX"].append(trX)
        st["trX2"].append(trX2)
        st["err"].append(err)
        if err < tol:
            status = "converged"
            break
        if stall_arm > 0:
            if abs(trX - trX2) < stall_arm:
                armed = True
            if armed and it >= 2 and err >= stall_ratio * st["err"][it - 2]:
                status = "stalled"
                break
        if it >= max_iter:
            break
        up = abs(2.0 * trX - trX2 - nocc) < abs(trX2 - nocc)
        st["branch"].append("2X-X2" if up else "X2")
        X = backend.update(X, r0, B, up, tau)
        it += 1
    st["iterations"] = it
    st["status"] = status
    return X, st


class GPUBlockOps:
    """Block operations through the CUDA library (FP64, full product rows): the block's
    Gershgorin bounds and X0, the traces of X (trX and ||X||_F^2 = tr X^2 for a symmetric
    X, the reading sp2_purify uses), and the thresholded product with the fused update
    against the block's rows plus the halo, placed in a matrix of the global row count."""

    def __init__(self, stream=None):
        from . import sp2ell as S
        self.S = S
        self.stream = stream

    def bounds(self, H, r0):
        return self.S.ellpack_gershgorin_block(H, r0, self.stream)

    def x0(self, H, r0, lo, hi, tau):
        X = self.S.Ellpack.empty(H.n, H.width + 32)
        self.S.sp2_x0_block(H, r0, lo, hi, tau, X, self.stream)
        return X

    def width(self, X):
        return X.width

    def widen(self, X, w):
        if X.width >= w:
            return X
        Y = self.S.Ellpack.empty(X.n, w)
        self.S.ellpack_copy(X, Y, self.stream)
        return Y

    def arrays(self, X):
        return X.idx, X.val, X.nnz

    def halo_requests(self, X, r0, r1, bounds):
        """{owner rank: device tensor of the rows it must send}, from the library's halo list."""
        import torch
        rows = self.S.ellpack_halo_rows(X, r0, bounds[-1], self.stream).to(torch.int64)
        cut = torch.searchsorted(rows, torch.tensor(bounds, dtype=torch.int64, device=rows.device)).cpu().tolist()
        return {q: rows[cut[q]:cut[q + 1]] for q in range(len(bounds) - 1) if cut[q + 1] > cut[q]}

    def extended(self, X, r0, n, halo):
        """A matrix of n rows holding the block's rows and the halo rows at their global
        positions (other rows empty)."""
        import torch
        B = self.S.Ellpack.empty(n, X.width)
        B.nnz.zero_()
        B.idx[r0:r0 + X.n] = X.idx
        B.val[r0:r0 + X.n] = X.val
        B.nnz[r0:r0 + X.n] = X.nnz
        rows, hi, hv, hn = halo
        if rows.numel():
            B.idx[rows] = hi
            B.val[rows] = hv
            B.nnz[rows] = hn
        torch.cuda.synchronize()
        return B

    def trace_parts(self, X, r0, B):
        tr, fro = self.S.ellpack_stats_block(X, r0, self.stream)
        return [tr], [fro]

    def update(self, X, r0, B, up, tau):
        """The block's product with the update, sized as sp2_purify sizes it (4x the longest row
        of X, at least 64, grown to the exact length on overflow) and then cut to its longest
        row, so that widths follow the rows and not the guesses."""
        S = self.S
        alpha, beta = (-1.0, 2.0) if up else (1.0, 0.0)
        longest = int(X.nnz.max().item()) if X.n else 0
        w = min(B.n, max(64, ((4 * longest + 31) // 32) * 32))
        while True:
            Y = S.Ellpack.empty(X.n, w)
            rc, req, _, _ = S.ellpack_multiply_block(X, r0, B, X if up else None, Y, alpha, beta, tau,
                                                     stream=self.stream, raise_on_overflow=False)
            if rc == 0:
                break
            w = min(B.n, ((req + 31) // 32) * 32)
        tight = max(32, ((req + 31) // 32) * 32)
        if tight < Y.width:
            Z = S.Ellpack.empty(X.n, tight)
            S.ellpack_copy(Y, Z, self.stream)
            Y = Z
        return Y
