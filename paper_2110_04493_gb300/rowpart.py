"""Row-partitioned squaring steps across ranks (one process per GPU): the host logic.

A squaring T~ = 2 T + T T (Eq. 4.15) followed by Algorithm 4.1 splits by rows:

* rank r owns the rows [b_r, b_{r+1}) of T^_k, a contiguous block chosen so that the blocks'
  product work (sum over k in row i of nnz(T_k), the scalar products of row i) is balanced;
* row i of T~ needs the rows T_k for every column k of row i: the rank's own rows plus a halo
  of rows owned by other ranks, which are exchanged before each squaring (the only data-path
  exchange of the step);
* Algorithm 4.1's thresholds are global: each pass sums the rank's dropped squares and the sum
  is all-reduced, so every rank follows the same threshold sequence; the relative threshold
  (||I + T~||_F) is an all-reduce of the ranks' partial sums as well;
* the filtered block stays on its rank; its place in the global CSR (row-pointer offset) is an
  exclusive scan of the ranks' kept counts.

The local arithmetic (the block's sparse product, one reduction pass, the compaction, the
partial norm) is supplied by a `LocalOps` object: `LibraryOps` runs it in libsexpm's CUDA
kernels; the collectives are torch.distributed calls on the given process group.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

# A row block in global coordinates: rows [r0, r1) of an n x n matrix, local row pointers
# (rp[0] = 0, r1 - r0 + 1 entries), global column indices.
Block = Tuple[int, int, int, np.ndarray, np.ndarray, np.ndarray]  # (n, r0, r1, rp, col, val)


# ------------------------------------------------------------------ partition and halo

def row_work(row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """Scalar products of each row of T T: sum over the columns k of row i of nnz(row k)."""
    lens = np.diff(row_ptr)
    w = lens[col].astype(np.int64)
    out = np.zeros(len(lens), dtype=np.int64)
    rows = np.repeat(np.arange(len(lens)), lens)
    np.add.at(out, rows, w)
    return out


def balanced_row_blocks(work: np.ndarray, world: int) -> np.ndarray:
    """Boundaries b_0 = 0 <= b_1 <= .. <= b_world = n of contiguous row blocks whose summed work
    is as even as a cut at row boundaries allows (each cut at the first row where the prefix
    of the work reaches r / world of the total, plus one so no row is split)."""
    n = len(work)
    pre = np.concatenate([[0], np.cumsum(work, dtype=np.int64)])
    total = pre[-1]
    b = [0]
    for r in range(1, world):
        target = total * r / world
        cut = int(np.searchsorted(pre, target, side="left"))
        b.append(min(max(cut, b[-1]), n))
    b.append(n)
    return np.asarray(b, dtype=np.int64)


def halo_rows(block: Block) -> np.ndarray:
    """Rows outside the block that its product rows read (columns of its rows outside [r0, r1))."""
    n, r0, r1, rp, col, val = block
    c = np.unique(col)
    return c[(c < r0) | (c >= r1)]


def owner_of(rows: np.ndarray, bounds: np.ndarray) -> np.ndarray:
    """Rank owning each row."""
    return np.searchsorted(bounds, rows, side="right") - 1


def split_requests(rows: np.ndarray, bounds: np.ndarray, world: int) -> List[np.ndarray]:
    """The halo rows grouped by their owning rank."""
    own = owner_of(rows, bounds)
    return [rows[own == p] for p in range(world)]


def rows_of_block(block: Block, rows: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """CSR slice (lengths, col, val) of the given global rows of a block (all inside it)."""
    n, r0, r1, rp, col, val = block
    loc = rows - r0
    lens = (rp[loc + 1] - rp[loc]).astype(np.int64)
    idx = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in loc]) if len(loc) else np.zeros(0, dtype=np.int64)
    return lens, col[idx], val[idx]


def assemble_operand(block: Block, halo: Sequence[Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]]
                     ) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The right operand of the block's product as an n x n CSR: the block's own rows plus the
    received halo rows (rows, lengths, col, val per peer); every other row is empty."""
    n, r0, r1, rp, col, val = block
    lens = np.zeros(n, dtype=np.int64)
    lens[r0:r1] = np.diff(rp)
    parts = {}
    for rows, rl, rc, rv in halo:
        lens[rows] = rl
        off = np.concatenate([[0], np.cumsum(rl)])
        for k, i in enumerate(rows):
            parts[int(i)] = (rc[off[k]:off[k + 1]], rv[off[k]:off[k + 1]])
    out_rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    out_c = np.empty(out_rp[-1], dtype=np.int32)
    out_v = np.empty(out_rp[-1], dtype=np.float64)
    out_c[out_rp[r0]:out_rp[r1]] = col
    out_v[out_rp[r0]:out_rp[r1]] = val
    for i, (c, v) in parts.items():
        out_c[out_rp[i]:out_rp[i + 1]] = c
        out_v[out_rp[i]:out_rp[i + 1]] = v
    return out_rp, out_c, out_v


def block_as_matrix(block: Block) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The block as an n x n CSR whose rows outside [r0, r1) are empty."""
    n, r0, r1, rp, col, val = block
    full = np.zeros(n + 1, dtype=np.int64)
    full[r0 + 1:r1 + 1] = rp[1:]
    full[r1 + 1:] = rp[-1]
    return full, col, val


def matrix_rows(n: int, r0: int, r1: int, rp: np.ndarray, col: np.ndarray, val: np.ndarray) -> Block:
    """Rows [r0, r1) of an n x n CSR as a block."""
    a, b = int(rp[r0]), int(rp[r1])
    return (n, r0, r1, (rp[r0:r1 + 1] - a).astype(np.int64), col[a:b].copy(), val[a:b].copy())


# ------------------------------------------------------------------ collectives

def _comm_device(group=None) -> str:
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def allreduce_sum(x: float, group=None) -> float:
    """Sum of a float over the ranks of the group (every rank receives it)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_comm_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return float(t.item())


def exclusive_offset(count: int, group=None) -> Tuple[int, int]:
    """(sum of count over the lower ranks, sum over all ranks): the place of this rank's kept
    entries in the global CSR."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    t = torch.tensor([count], dtype=torch.int64, device=_comm_device(group))
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    vals = [int(x.item()) for x in out]
    return sum(vals[:me]), sum(vals)


def exchange_halo(block: Block, requests: List[np.ndarray], group=None
                  ) -> List[Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]]:
    """Sends every peer the rows of this block it asks for and receives the rows this rank asked
    for (requests[p]: rows wanted from rank p).  Returns (rows, lengths, col, val) per peer."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    dev = _comm_device(group)
    counts = torch.tensor([len(r) for r in requests], dtype=torch.int64, device=dev)
    table = [torch.zeros_like(counts) for _ in range(world)]
    dist.all_gather(table, counts, group=group)
    asked = [int(table[p][me].item()) for p in range(world)]  # rows peer p wants from me

    def send_recv(send_list, recv_shapes, dtype):
        # every receive is posted before any send, then all are awaited (no ordering deadlock)
        works = []
        recv = {}
        for p in range(world):
            if p != me and recv_shapes[p]:
                recv[p] = torch.empty(recv_shapes[p], dtype=dtype, device=dev)
                works.append(dist.irecv(recv[p], src=p, group=group))
        for p in range(world):
            if p != me and send_list[p] is not None and send_list[p].numel():
                works.append(dist.isend(send_list[p], dst=p, group=group))
        for w in works:
            w.wait()
        return recv

    # 1. the row lists
    req_t = [torch.from_numpy(np.ascontiguousarray(r, dtype=np.int64)).to(dev) if p != me else None
             for p, r in enumerate(requests)]
    wanted = send_recv(req_t, [asked[p] if p != me else 0 for p in range(world)], torch.int64)
    # 2. lengths of the requested rows, then their entries
    slices = {}
    lens_t = [None] * world
    for p in range(world):
        if p == me or not asked[p]:
            continue
        rows = wanted[p].cpu().numpy()
        slices[p] = rows_of_block(block, rows)
        lens_t[p] = torch.from_numpy(slices[p][0]).to(dev)
    got_lens = send_recv(lens_t, [len(requests[p]) if p != me else 0 for p in range(world)], torch.int64)
    tot_in = [int(got_lens[p].sum().item()) if p in got_lens else 0 for p in range(world)]
    col_t = [torch.from_numpy(np.ascontiguousarray(slices[p][1], dtype=np.int32)).to(dev) if p in slices else None
             for p in range(world)]
    val_t = [torch.from_numpy(np.ascontiguousarray(slices[p][2], dtype=np.float64)).to(dev) if p in slices else None
             for p in range(world)]
    got_col = send_recv(col_t, tot_in, torch.int32)
    got_val = send_recv(val_t, tot_in, torch.float64)
    out = []
    for p in range(world):
        if p == me or not len(requests[p]):
            continue
        out.append((np.asarray(requests[p], dtype=np.int64), got_lens[p].cpu().numpy(),
                    got_col[p].cpu().numpy() if p in got_col else np.zeros(0, np.int32),
                    got_val[p].cpu().numpy() if p in got_val else np.zeros(0)))
    return out


def alg41_distributed(local_sum: Callable[[float], float], eps_g: float, e_r: float, max_iters: int = 100,
                      group=None) -> Tuple[float, int, float]:
    """Algorithm 4.1 with the reduction split over ranks: t_0 = eps_g, b_j = sqrt(sum over ranks of
    the local sums of v^2 over |v| <= t_j), t_{j+1} = eps_g t_j / b_j, until b_j <= eps_g (1 + e_r).
    Every rank computes the same sequence.  Returns (t, passes, b)."""
    m = 1.0
    b = math.inf
    t = eps_g
    it = 0
    while b > eps_g * (1.0 + e_r):
        if it >= max_iters:
            raise RuntimeError(f"Algorithm 4.1 did not converge within {max_iters} passes")
        t = eps_g / m
        b = math.sqrt(allreduce_sum(local_sum(t), group))
        m = b / t
        it += 1
    return t, it, b


# ------------------------------------------------------------------ one squaring step

class LocalOps:
    """The local arithmetic of a row-partitioned squaring.  Matrices are n x n CSR triples
    (row_ptr, col, val) whose rows outside the rank's block are empty."""

    def product(self, A, B):
        """(A B) + 2 A: rows of T~ = 2 T + T T for the block A, with B = the block plus its halo."""
        raise NotImplementedError

    def norm2_I_plus_rows(self, X, r0: int, r1: int) -> float:
        """sum over rows r0..r1-1 of sum_j (delta_ij + x_ij)^2."""
        raise NotImplementedError

    def pass_sum(self, X, t: float) -> float:
        """sum of v^2 over the stored entries of X with |v| <= t."""
        raise NotImplementedError

    def apply(self, X, t: float):
        """The entries of X with |v| > t (CSR triple)."""
        raise NotImplementedError


class LibraryOps(LocalOps):
    """LocalOps on this rank's GPU through libsexpm's C ABI (sexpm_spgemm, sexpm_filter_pass,
    sexpm_filter_apply, sexpm_norm2_I_plus_rows)."""

    def __init__(self, n: int):
        from . import sexpm
        self.sx = sexpm
        self.n = n

    def _dev(self, X):
        import torch
        rp, ci, v = X
        return (torch.from_numpy(np.asarray(rp, dtype=np.int64)).cuda(),
                torch.from_numpy(np.asarray(ci, dtype=np.int32)).cuda(),
                torch.from_numpy(np.asarray(v, dtype=np.float64)).cuda(), self.n)

    @staticmethod
    def _host(t):
        return tuple(x.cpu().numpy() for x in t)

    def product(self, A, B):
        dA, dB = self._dev(A), self._dev(B)
        out, _ = self.sx.spgemm(dA, dB, dA, div=1.0, beta=2.0)
        return self._host(out)

    def norm2_I_plus_rows(self, X, r0, r1):
        return self.sx.norm2_I_plus_rows(self._dev(X), r0, r1)

    def pass_sum(self, X, t):
        return self.sx.filter_pass(self._dev(X), t)[0]

    def apply(self, X, t):
        return self._host(self.sx.filter_apply(self._dev(X), t))


def square_step(block: Block, bounds: np.ndarray, k: int, a: float, r0_bound: float, e_r: float, ops: LocalOps,
                square_scale: bool = True, max_iters: int = 100, group=None):
    """One filtered squaring T^_k = filter(2 T^_{k-1} + T^_{k-1}^2) on this rank's row block
    (Eq. 4.15, Algorithm 4.1 with eps_g = a 2^k r_0 ||I + T~_k||_F, or a 2^k r_0 when
    square_scale is False).  Every rank calls it with its own block and the same bounds.
    Returns (the new block, {"eps_g", "t", "iters", "b", "nnz_raw", "nnz"}) with nnz_* summed
    over ranks."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n, b0, b1 = block[0], block[1], block[2]
    requests = split_requests(halo_rows(block), bounds, world)
    received = exchange_halo(block, requests, group)
    B = assemble_operand(block, received)
    A = block_as_matrix(block)
    Tt = ops.product(A, B)
    normF = 1.0
    if square_scale:
        normF = math.sqrt(max(allreduce_sum(ops.norm2_I_plus_rows(Tt, b0, b1), group), 0.0))
    eps_g = a * math.ldexp(r0_bound, k) * normF
    t, it, bnorm = alg41_distributed(lambda th: ops.pass_sum(Tt, th), eps_g, e_r, max_iters, group)
    Tn = ops.apply(Tt, t)
    new = matrix_rows(n, b0, b1, *Tn)
    _, raw_total = exclusive_offset(int(Tt[0][-1]), group)
    _, kept_total = exclusive_offset(int(new[3][-1]), group)
    return new, {"eps_g": eps_g, "t": t, "iters": it, "b": bnorm, "nnz_raw": raw_total, "nnz": kept_total}


def gather_blocks(block: Block, group=None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The whole matrix from every rank's block (in rank order), as a CSR triple on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, block, group=group)
    n = parts[0][0]
    lens = np.zeros(n, dtype=np.int64)
    cols, vals = [], []
    for (_, r0, r1, rp, col, val) in parts:
        lens[r0:r1] = np.diff(rp)
        cols.append(col)
        vals.append(val)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return rp, np.concatenate(cols).astype(np.int32), np.concatenate(vals)
