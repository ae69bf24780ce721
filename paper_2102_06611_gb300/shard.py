"""One population-annealing run split over several shards by contiguous ranges of replica
slots (arXiv:2102.06611, Sec. II: one population of R_i replicas, normalised once per step by
Eqs. Q and taus).

Each shard sweeps and measures its own replicas.  Once per temperature step the shards
exchange:
  1. summaries (level histogram, exact sums, family edges): an all-gather, after which every
     shard holds the whole population's histogram and sums (pa_shard_combine);
  2. their children counts c_s after resampling: an all-gather whose exclusive scan gives the
     children of shard s the global slots [o_s, o_s + c_s);
  3. the children themselves: the new population is re-split into contiguous ranges of
     (nearly) equal size and each shard writes the children that fall into a range straight
     into the owner's buffers (its own, another on the same device, or a staging area sent
     point-to-point), so no shard ever holds more than its parents and its new share.
Random numbers are keyed by the global slot, so the result is the one population held whole
would give, for any number of shards.

A shard is an *engine*: the GPU engine (`GpuShard`, the C ABI's pa_shard_* calls on this
process's device) or any object with the same methods.  A *transport* carries the exchanges:
`LocalTransport` for several shards held by one process (e.g. on one GPU), `DistTransport`
for one shard per torch.distributed rank (NCCL between GPUs, gloo between CPU processes).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _check, _lib, default_capacity


# ------------------------------------------------------------------------------ plan
def split(R: int, n_shards: int, shard: int) -> tuple[int, int]:
    """Slot range [lo, hi) of `shard` when R replicas are split into n_shards contiguous ranges
    of nearly equal size."""
    return (shard * R) // n_shards, ((shard + 1) * R) // n_shards


@dataclass
class Transfer:
    src: int        # shard whose parents produce the children
    src_off: int    # first child, local child index in src (tree order)
    dst: int        # shard receiving them (into its non-current buffers)
    dst_off: int    # local index in dst's new population
    count: int


@dataclass
class Plan:
    R_total: int
    lo: list[int]          # new slot base of each shard
    size: list[int]        # new local size of each shard
    transfers: list[Transfer]


def rebalance_plan(totals: list[int]) -> Plan:
    """Children of shard s occupy the global slots [o_s, o_s + c_s), o = exclusive scan of the
    totals c (tree order across shards); the new population is split evenly and every
    non-empty intersection of a child range with a new range is one transfer."""
    P = len(totals)
    offs, o = [], 0
    for c in totals:
        offs.append(o)
        o += int(c)
    R = o
    lo = [split(R, P, t)[0] for t in range(P)]
    hi = [split(R, P, t)[1] for t in range(P)]
    transfers = []
    for s in range(P):
        a, b = offs[s], offs[s] + int(totals[s])
        for t in range(P):
            x, y = max(a, lo[t]), min(b, hi[t])
            if x < y:
                transfers.append(Transfer(s, x - a, t, x - lo[t], y - x))
    return Plan(R, lo, [hi[t] - lo[t] for t in range(P)], transfers)


# ------------------------------------------------------------------------------ transports
class LocalTransport:
    """All shards in this process (engines indexed by shard number)."""

    def all_gather(self, local: dict[int, torch.Tensor], n_shards: int) -> torch.Tensor:
        return torch.stack([local[s] for s in range(n_shards)])

    def all_gather_ints(self, local: dict[int, int], n_shards: int) -> list[int]:
        return [int(local[s]) for s in range(n_shards)]

    def move(self, plan: Plan, engines: dict) -> None:
        for tr in plan.transfers:  # children written straight into the owner's buffers
            engines[tr.src].copy_children(tr.src_off, tr.count, engines[tr.dst].views(tr.dst_off, tr.count))


class DistTransport:
    """One or more shards per torch.distributed rank; shard s lives on rank owner(s)."""

    def __init__(self, group=None, shards_per_rank: int = 1):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.k = shards_per_rank

    def owner(self, shard: int) -> int:
        return shard // self.k

    def all_gather(self, local: dict[int, torch.Tensor], n_shards: int) -> torch.Tensor:
        mine = torch.stack([local[s] for s in sorted(local)])
        parts = [torch.empty_like(mine) for _ in range(n_shards // self.k)]
        self.dist.all_gather(parts, mine, group=self.group)
        return torch.cat(parts)

    def all_gather_ints(self, local: dict[int, int], n_shards: int) -> list[int]:
        dev = torch.device("cuda", torch.cuda.current_device()) if self.dist.get_backend(self.group) == "nccl" \
            else torch.device("cpu")
        mine = torch.tensor([int(local[s]) for s in sorted(local)], dtype=torch.int64, device=dev)
        parts = [torch.empty_like(mine) for _ in range(n_shards // self.k)]
        self.dist.all_gather(parts, mine, group=self.group)
        return [int(v) for v in torch.cat(parts).tolist()]

    def move(self, plan: Plan, engines: dict) -> None:
        me = self.dist.get_rank(self.group)
        ops, tags, keep = [], [], []
        for i, tr in enumerate(plan.transfers):
            src_here, dst_here = self.owner(tr.src) == me, self.owner(tr.dst) == me
            if src_here and dst_here:
                engines[tr.src].copy_children(tr.src_off, tr.count, engines[tr.dst].views(tr.dst_off, tr.count))
            elif src_here:
                buf = engines[tr.src].staging(tr.count)
                engines[tr.src].copy_children(tr.src_off, tr.count, buf)
                keep.append(buf)
                for k, v in enumerate(buf):
                    ops.append(self.dist.P2POp(self.dist.isend, v, self.owner(tr.dst), self.group))
                    tags.append(4 * i + k)
            elif dst_here:
                for k, v in enumerate(engines[tr.dst].views(tr.dst_off, tr.count)):
                    ops.append(self.dist.P2POp(self.dist.irecv, v, self.owner(tr.src), self.group))
                    tags.append(4 * i + k)
        if ops:
            if self.dist.get_backend(self.group) == "nccl":
                reqs = self.dist.batch_isend_irecv(ops)  # one NCCL group: no ordering deadlock
            else:  # gloo: tagged messages, the tag naming the transfer and the array
                reqs = [op.op(op.tensor, op.peer, group=self.group, tag=t) for op, t in zip(ops, tags)]
            for r in reqs:
                r.wait()
        del keep


# ------------------------------------------------------------------------------ GPU engine
class GpuShard:
    """One shard on this process's GPU through the C ABI (pa_shard_*).  Buffers are torch
    tensors; the library allocates nothing."""

    def __init__(self, L: int, R: int, seed: int, slot_base: int, R_local: int, capacity: int,
                 resample: str = "nearest", update: str = "metropolis", device=None,
                 stream: torch.cuda.Stream | None = None):
        self.lib = _lib.lib()
        self.L, self.N, self.R = int(L), int(L) * int(L), int(R)
        kind = {"nearest": _lib.PA_RESAMPLE_NEAREST, "poisson": _lib.PA_RESAMPLE_POISSON,
                "multinomial": _lib.PA_RESAMPLE_MULTINOMIAL}[resample]
        upd = {"metropolis": _lib.PA_UPDATE_METROPOLIS, "heatbath": _lib.PA_UPDATE_HEATBATH}[update]
        self.device = torch.device(device if device is not None else "cuda")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.capacity = int(capacity)
        self.cfg = _lib.pa_config(L=self.L, resample=kind, R=self.R, capacity=self.capacity, seed=int(seed),
                                  update=upd)
        sized = _lib.pa_config(L=self.L, resample=kind, R=self.capacity, capacity=self.capacity, seed=int(seed),
                               update=upd)
        sizes = _lib.pa_sizes()
        _check(self.lib, None, self.lib.pa_query_sizes(ctypes.byref(sized), ctypes.byref(sizes)))
        self.bpr = sizes.bytes_per_replica
        dev = self.device
        self.spins = [torch.empty(sizes.spin_bytes, dtype=torch.uint8, device=dev) for _ in range(2)]
        self.level = [torch.empty(self.capacity, dtype=torch.int32, device=dev) for _ in range(2)]
        self.mag = [torch.empty(self.capacity, dtype=torch.int32, device=dev) for _ in range(2)]
        self.fam = [torch.empty(self.capacity, dtype=torch.int32, device=dev) for _ in range(2)]
        self.work = torch.empty(sizes.work_bytes, dtype=torch.uint8, device=dev)
        bufs = _lib.pa_buffers()
        for b in range(2):
            bufs.spins[b] = self.spins[b].data_ptr()
            bufs.level[b] = self.level[b].data_ptr()
            bufs.mag[b] = self.mag[b].data_ptr()
            bufs.fam[b] = self.fam[b].data_ptr()
        bufs.work = self.work.data_ptr()
        self._bufs = bufs
        self.V = int(self.lib.pa_shard_summary_len(self.L))
        self._summary = torch.zeros(self.V, dtype=torch.int64, device=dev)
        ctx = ctypes.c_void_p()
        with torch.cuda.device(dev):
            st = self.lib.pa_shard_init(ctypes.byref(self.cfg), int(slot_base), int(R_local), ctypes.byref(bufs),
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        _check(self.lib, None, st)
        self.ctx = ctx
        self._all = None
        self.cur = 0  # index of the current buffers (mirrors the context's, see layout())

    def summary(self) -> torch.Tensor:
        _check(self.lib, self.ctx, self.lib.pa_shard_summary(self.ctx, ctypes.c_void_p(self._summary.data_ptr())))
        return self._summary

    def combine(self, all_summaries: torch.Tensor) -> None:
        self._all = all_summaries.to(self.device).contiguous()  # kept alive until the kernel has run
        _check(self.lib, self.ctx, self.lib.pa_shard_combine(self.ctx, ctypes.c_void_p(self._all.data_ptr()),
                                                             int(self._all.shape[0])))

    def resample(self, beta: float) -> None:
        """Copy numbers of this shard's parents; local_size() is then its number of children."""
        _check(self.lib, self.ctx, self.lib.pa_resample(self.ctx, float(beta)))

    def layout(self) -> tuple[int, int, int]:
        cur, R, base = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(self.lib, self.ctx, self.lib.pa_shard_layout(self.ctx, ctypes.byref(cur), ctypes.byref(R),
                                                            ctypes.byref(base)))
        return cur.value, R.value, base.value

    def local_size(self) -> int:
        return self.layout()[1]

    def views(self, off: int, count: int):
        """(spin bytes, level, magnetisation, family id) of replicas [off, off + count) of the
        non-current buffers, where the next population is assembled."""
        b = self.cur ^ 1
        return (self.spins[b][off * self.bpr:(off + count) * self.bpr], self.level[b][off:off + count],
                self.mag[b][off:off + count], self.fam[b][off:off + count])

    def staging(self, count: int):
        """Fresh device arrays for `count` children to be sent to another shard."""
        return (torch.empty(count * self.bpr, dtype=torch.uint8, device=self.device),
                torch.empty(count, dtype=torch.int32, device=self.device),
                torch.empty(count, dtype=torch.int32, device=self.device),
                torch.empty(count, dtype=torch.int32, device=self.device))

    def copy_children(self, first: int, count: int, dst) -> None:
        """Children [first, first + count) of the last resampling into the arrays dst (as views()
        returns them: spin bytes, level, magnetisation, family id)."""
        sp, lv, mg, fm = dst
        _check(self.lib, self.ctx, self.lib.pa_shard_copy(self.ctx, int(first), int(count),
                                                          ctypes.c_void_p(sp.data_ptr()), ctypes.c_void_p(lv.data_ptr()),
                                                          ctypes.c_void_p(mg.data_ptr()), ctypes.c_void_p(fm.data_ptr())))

    def adopt(self, R_local: int, slot_base: int) -> None:
        _check(self.lib, self.ctx, self.lib.pa_shard_adopt(self.ctx, int(R_local), int(slot_base)))
        self.cur ^= 1

    def anneal_step(self, theta: int) -> None:
        _check(self.lib, self.ctx, self.lib.pa_anneal_step(self.ctx, int(theta)))

    def observables(self) -> dict:
        o = _lib.pa_obs()
        _check(self.lib, self.ctx, self.lib.pa_observables(self.ctx, ctypes.byref(o)))
        return o.as_dict()

    def record(self, dst: torch.Tensor) -> None:
        _check(self.lib, self.ctx, self.lib.pa_record(self.ctx, ctypes.c_void_p(dst.data_ptr())))

    # testing accessors (synchronising, host results)
    def histogram(self):
        import numpy as np
        h = np.zeros(self.N + 1, np.int32)
        _check(self.lib, self.ctx, self.lib.pa_histogram(self.ctx, h.ctypes.data))
        return h

    def hashes(self):
        import numpy as np
        R = self.local_size()
        out = np.zeros(max(R, 1), np.uint64)
        _check(self.lib, self.ctx, self.lib.pa_hashes(self.ctx, out.ctypes.data))
        return out[:R]

    def replicas(self):
        import numpy as np
        R = self.local_size()
        lv, mg, fm = (np.zeros(max(R, 1), np.int32) for _ in range(3))
        _check(self.lib, self.ctx, self.lib.pa_replicas(self.ctx, lv.ctypes.data, mg.ctypes.data, fm.ctypes.data))
        return lv[:R], mg[:R], fm[:R]

    def copy_counts(self):
        import numpy as np
        out = np.zeros(self.capacity, np.int32)
        n = ctypes.c_longlong()
        _check(self.lib, self.ctx, self.lib.pa_copy_counts(self.ctx, out.ctypes.data, ctypes.byref(n)))
        return out[: n.value].copy()

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.pa_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------ driver
class ShardedRun:
    """The shards of one population held by this process (`engines`: shard number -> engine)
    and the transport between all n_shards shards.  Every process calls the same methods in
    the same order."""

    def __init__(self, engines: dict, n_shards: int, transport):
        self.engines = dict(engines)
        self.P = int(n_shards)
        self.transport = transport
        self.plan: Plan | None = None
        self._exchange_summaries()

    def _exchange_summaries(self) -> None:
        local = {s: e.summary() for s, e in self.engines.items()}
        allv = self.transport.all_gather(local, self.P)
        for e in self.engines.values():
            e.combine(allv)

    def resample(self, beta: float) -> Plan:
        """Step 2 over all shards: local copy numbers and children, then the re-split."""
        for e in self.engines.values():
            e.resample(beta)
        totals = self.transport.all_gather_ints({s: e.local_size() for s, e in self.engines.items()}, self.P)
        plan = rebalance_plan(totals)
        self.transport.move(plan, self.engines)
        for s, e in self.engines.items():
            e.adopt(plan.size[s], plan.lo[s])
        self.plan = plan
        return plan

    def anneal_step(self, theta: int) -> None:
        """Step 3 on every shard, then the summaries of the new measurement."""
        for e in self.engines.values():
            e.anneal_step(theta)
        self._exchange_summaries()

    def observables(self) -> dict:
        """Step 4 of the whole population (identical on every shard)."""
        return next(iter(self.engines.values())).observables()


def shard_capacity(R: int, n_shards: int) -> int:
    """Buffer capacity of one shard: its share of a population whose size fluctuates by
    ~sqrt(R) (the re-split keeps shares within one replica of each other)."""
    import math
    return -(-R // n_shards) + int(math.ceil(10.0 * math.sqrt(R) / n_shards)) + 64


def gpu_shards(L: int, R: int, seed: int, shards: list[int], n_shards: int, resample: str = "nearest",
               update: str = "metropolis", device=None, stream=None, capacity: int | None = None) -> dict:
    """GPU engines for the listed shards of the simple-sampling population of step 1."""
    cap = capacity if capacity is not None else shard_capacity(R, n_shards)
    out = {}
    for s in shards:
        lo, hi = split(R, n_shards, s)
        out[s] = GpuShard(L, R, seed, lo, hi - lo, cap, resample=resample, update=update, device=device, stream=stream)
    return out
