"""A CPU shard engine for the sharded-run driver (paper_2102_06611_gb300.shard), built from the
oracle's per-replica primitives: test infrastructure only.  It lets the driver's exchange
protocol (summaries, the scan of children counts, the re-split of the new population) run on
gloo ranks without a GPU, against the oracle's single population as the reference.

The method's arithmetic stays in the oracle: simple sampling (init_replica), sweeps
(sweep_replica), energies (energy_mag), the copy numbers of a shard's parents from the whole
histogram (resample_shard, Sec. II Eqs. Q and taus; multinomial draws also take the histogram
of the shards before this one) and the observables (observables_from_sums,
Sec. III).  This file only holds the population arrays, moves replicas, and merges family runs
across shard boundaries."""
from __future__ import annotations

import math

import numpy as np
import torch

import oracle

EXTRA = 16


class OracleShard:
    def __init__(self, L, R, seed, slot_base, R_local, capacity, kind=oracle.NEAREST, update=oracle.METROPOLIS):
        self.L, self.N, self.R, self.seed, self.kind, self.update = L, L * L, R, seed, kind, update
        self.capacity = capacity
        self.spins = [torch.zeros((capacity, L * L), dtype=torch.int8) for _ in range(2)]
        self.level = [torch.zeros(capacity, dtype=torch.int32) for _ in range(2)]
        self.mag = [torch.zeros(capacity, dtype=torch.int32) for _ in range(2)]
        self.fam = [torch.zeros(capacity, dtype=torch.int32) for _ in range(2)]
        self.cur, self.n, self.base = 0, R_local, slot_base
        for j in range(R_local):
            self.spins[0][j] = torch.from_numpy(oracle.init_replica(L, seed, slot_base + j))
            self.fam[0][j] = slot_base + j
        self._measure()
        self.step, self.beta, self.dbeta, self.lnQ, self.sum_lnQ, self.sum_lnR = 0, 0.0, 0.0, 0.0, 0.0, 0.0
        self.t_done, self.theta_last = 0, 0
        self.counts = np.zeros(0, np.int32)
        self.children = None
        self.glob = None

    def _measure(self):
        c = self.cur
        for j in range(self.n):
            E, M = oracle.energy_mag(self.L, self.spins[c][j].numpy())
            self.level[c][j] = (E + 2 * self.N) // 4
            self.mag[c][j] = M

    def _arrays(self):
        c = self.cur
        lv = self.level[c][: self.n].numpy()
        return lv, 4 * lv.astype(np.int64) - 2 * self.N, self.mag[c][: self.n].numpy(), self.fam[c][: self.n].numpy()

    def summary(self):
        lv, E, M, F = self._arrays()
        out = np.zeros(self.N + 1 + EXTRA, np.int64)
        out[: self.N + 1] = np.bincount(lv, minlength=self.N + 1)
        x = out[self.N + 1:]
        x[0] = self.n
        sums = oracle.population_sums(E, M, F)
        x[1], x[2] = sums[2], sums[3]
        if self.n:
            first = int(np.argmax(F != F[0])) if np.any(F != F[0]) else self.n
            last = int(np.argmax(F[::-1] != F[-1])) if np.any(F != F[-1]) else self.n
            x[8], x[9], x[10], x[11] = F[0], first, F[-1], last
            x[12], x[13] = sums[4], sums[5]
        return torch.from_numpy(out)

    def combine(self, allv):
        a = allv.numpy()
        N1 = self.N + 1
        hist = a[:, :N1].sum(axis=0)
        R = int(a[:, N1].sum())
        # levels of the parents in the shards before this one (rows in slot order): the
        # multinomial draws need their weight sum
        ends = np.cumsum(a[:, N1])
        before = a[ends <= self.base, :N1].sum(axis=0)
        # family runs: walk the shards' run lists in slot order; a shard contributes its first
        # run, its inner runs (count, sum of squared lengths) and its last run, and a run that
        # continues across a boundary is joined
        runs = []  # ("run", id, length) or ("inner", count, sum of length^2)
        for x in a[:, N1:]:
            if x[0] <= 0:
                continue
            pieces = [("run", int(x[8]), int(x[9]))]
            if x[12] > 1:
                pieces += [("inner", int(x[12]) - 2, int(x[13] - x[9] ** 2 - x[11] ** 2)),
                           ("run", int(x[10]), int(x[11]))]
            for p in pieces:
                if p[0] == "run" and runs and runs[-1][0] == "run" and runs[-1][1] == p[1]:
                    runs[-1] = ("run", p[1], runs[-1][2] + p[2])
                else:
                    runs.append(p)
        f = sum(1 if r[0] == "run" else r[1] for r in runs)
        s2 = sum(r[2] ** 2 if r[0] == "run" else r[2] for r in runs)
        sE = int((hist * (4 * np.arange(N1, dtype=np.int64) - 2 * self.N)).sum())
        sE2 = int((hist * (4 * np.arange(N1, dtype=np.int64) - 2 * self.N) ** 2).sum())
        self.glob = {"hist": hist, "R": R, "hist_before": before,
                     "isums": np.array([sE, sE2, a[:, N1 + 1].sum(), a[:, N1 + 2].sum(), f, s2], np.int64)}

    def resample(self, beta):
        """Copy numbers of this shard's parents from the whole histogram; the children are
        written by copy_children into the shards that own their slots."""
        g = self.glob
        lv, _, _, _ = self._arrays()
        self.step += 1
        st, counts, lnQ, R_new = oracle.resample_shard(self.L, self.R, g["hist"], g["R"], lv, self.base, self.beta,
                                                       beta, self.step, self.seed, self.kind,
                                                       hist_before=g["hist_before"])
        assert st == 0
        self.counts = counts
        self.children = np.repeat(np.arange(self.n), counts)   # parent of each child, tree order
        self.lnQ = lnQ
        self.sum_lnQ = self.sum_lnQ + lnQ
        self.sum_lnR = self.sum_lnR + math.log(g["R"] / self.R)
        self.dbeta = beta - self.beta
        self.beta = beta
        self.t_done = 0
        self.glob = None

    def local_size(self):
        return len(self.children) if self.children is not None else self.n

    def views(self, off, count):
        b = self.cur ^ 1
        return (self.spins[b][off:off + count], self.level[b][off:off + count], self.mag[b][off:off + count],
                self.fam[b][off:off + count])

    def staging(self, count):
        return (torch.zeros((count, self.N), dtype=torch.int8), torch.zeros(count, dtype=torch.int32),
                torch.zeros(count, dtype=torch.int32), torch.zeros(count, dtype=torch.int32))

    def copy_children(self, first, count, dst):
        idx = torch.from_numpy(self.children[first:first + count]).long()
        c = self.cur
        for src, d in zip((self.spins[c], self.level[c], self.mag[c], self.fam[c]), dst):
            d[:] = src[idx]

    def adopt(self, R_local, slot_base):
        self.cur ^= 1
        self.n, self.base = R_local, slot_base
        self.children = None

    def anneal_step(self, theta):
        c = self.cur
        for j in range(self.n):
            s = oracle.sweep_replica(self.L, self.seed, self.step, self.base + j, self.beta, theta,
                                     self.spins[c][j].numpy(), t0=self.t_done, update=self.update)
            self.spins[c][j] = torch.from_numpy(s)
        self.t_done += theta
        self.theta_last = theta
        self._measure()

    def observables(self):
        g = self.glob
        return oracle.observables_from_sums(self.N, g["R"], g["isums"], self.beta, self.dbeta, self.lnQ,
                                            self.sum_lnQ, self.sum_lnR, self.step, self.theta_last)

    def hashes(self):
        return np.array([oracle.replica_hash(self.L, self.spins[self.cur][j].numpy()) for j in range(self.n)],
                        np.uint64)

    def families(self):
        return self.fam[self.cur][: self.n].numpy().copy()
