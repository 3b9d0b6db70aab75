"""The z-slab decomposition's host logic, on CPU.

- partition / receivers: cuts keep the z layer inside the end slabs, every
  receiver is sampled by exactly one slab and injected by the one or two slabs
  that own its planes, local receiver z is exact;
- the march over 2 and 3 gloo ranks: a CPU stand-in for the step kernels (two
  field families updated from each other through staggered fourth-order z
  differences that reach two planes, receivers sampled and injected on two
  planes, zero outside the held planes) run slab by slab with DistExchange
  gives bitwise the traces and image of the same stand-in on the whole grid,
  with receivers on both sides of the cuts, and every rank assembles the
  whole traces and image exactly (sum all-reduces over disjoint parts) and the
  inner products' partial sums (one scalar all-reduce each).  A missing or misordered
  exchange, a wrong halo slice, or a receiver sampled twice or injected on the
  wrong slabs changes the result.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1709_02733_b300 import slabs, synth  # noqa: E402

NZ, NY, NX = 48, 3, 4
NPML = 4
C1, C2 = 9.0 / 8.0, -1.0 / 24.0


def _receivers(L=23, seed=3):
    rng = np.random.default_rng(seed)
    rec = np.stack([rng.uniform(0, NX - 2, L), rng.uniform(0, NY - 2, L), rng.uniform(0, NZ - 2, L)], 1)
    rec[0, 2] = NZ - 2          # on the last admissible plane
    rec[1, 2] = 20.0            # on a plane exactly
    rec[2, 2] = 23.5            # straddling the cut of two slabs (24)
    rec[3, 2] = 15.25           # and of three slabs (16, 32)
    rec[4, 2] = 31.75
    rec[5, 2] = 24.0            # on the cut plane of two slabs
    return rec.astype(np.float32)


# -- partition ----------------------------------------------------------------------

@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_partition_and_receivers(R):
    rec = _receivers()
    parts = slabs.partition(NZ, R, NPML)
    assert parts[0][0] == 0 and parts[-1][1] == NZ
    assert all(parts[r][1] == parts[r + 1][0] for r in range(R - 1))
    for lo, hi in parts[1:]:
        assert NPML + 4 <= lo <= NZ - NPML - 4
    k0 = slabs.receiver_planes(rec, NZ)
    sampled = np.zeros(len(rec), int)
    injected = np.zeros(len(rec), int)
    for r in range(R):
        s = slabs.layout(NZ, parts, r, rec)
        lo, hi = parts[r]
        sampled[s.rec_idx] += 1
        injected[s.inj_idx] += 1
        assert np.all((k0[s.rec_idx] >= lo) & (k0[s.rec_idx] < hi))
        assert np.all(((k0[s.inj_idx] >= lo) & (k0[s.inj_idx] < hi)) |
                      ((k0[s.inj_idx] + 1 >= lo) & (k0[s.inj_idx] + 1 < hi)))
        for idx, loc in ((s.rec_idx, s.rec_local), (s.inj_idx, s.inj_local)):
            assert np.all(np.diff(idx) > 0)
            # local z is exact: the same planes and weights as the whole grid
            z = loc[:, 2]
            assert np.array_equal(z + np.float32(s.zl), rec[idx, 2])
            kl = np.minimum(np.floor(z).astype(np.int64), s.nzl - 2)
            assert np.array_equal(kl + s.zl, k0[idx])
            assert np.array_equal(z - kl, rec[idx, 2] - k0[idx])
            assert np.all((kl >= 0) & (kl + 1 < s.nzl))
        assert s.zh - s.zl >= 5
    assert np.all(sampled == 1)
    straddle = np.isin(k0 + 1, [lo for lo, _ in parts[1:]])
    assert np.all(injected == 1 + straddle)
    assert straddle.any() == (R > 1)


def test_partition_skull_512():
    """The bench grid splits into up to 8 equal slabs."""
    for R in (2, 4, 8):
        parts = slabs.partition(512, R, 20)
        assert {hi - lo for lo, hi in parts} == {512 // R}


def test_partition_rejects_impossible():
    with pytest.raises(ValueError):
        slabs.partition(24, 2, 9)          # the cut would fall in the z layer's reach
    with pytest.raises(ValueError):
        slabs.partition(NZ, 7, 0)          # fewer than MIN_OWNED planes a slab


# -- the march with a CPU stand-in for the step kernels ------------------------------

def _dz_fwd(f):
    """Staggered fourth-order z difference at k + 1/2 (reach k-1 .. k+2), zero
    outside the held planes."""
    g = torch.nn.functional.pad(f, (0, 0, 0, 0, 1, 2))
    return C1 * (g[2:-1] - g[1:-2]) + C2 * (g[3:] - g[:-3])


def _dz_bwd(f):
    """At k - 1/2 (reach k-2 .. k+1)."""
    g = torch.nn.functional.pad(f, (0, 0, 0, 0, 2, 1))
    return C1 * (g[2:-1] - g[1:-2]) + C2 * (g[3:] - g[:-3])


class FakeGrid:
    """Nine float64 fields; the velocity half writes slots 0..2 from slots 3..8,
    the stress half slots 3..8 from slots 0..2, both with z differences that
    reach two planes up and down; receivers read / write slot 3 on planes k0,
    k0+1."""

    def __init__(self, nzl):
        self.shape = (nzl, NY, NX)
        self.f = torch.zeros((9,) + self.shape, dtype=torch.float64)

    def field_view(self, k):
        return self.f[k]

    def _taps(self):
        z = torch.as_tensor(self.rec[:, 2], dtype=torch.float64)
        k0 = torch.clamp(torch.floor(z).long(), max=self.shape[0] - 2)
        fz = z - k0
        x = torch.as_tensor(self.rec[:, 0]).long()
        y = torch.as_tensor(self.rec[:, 1]).long()
        return k0, fz, y, x

    def begin(self, adj, inp, rec, nsteps, out):
        self.f.zero_()
        self.adj, self.rec, self.nsteps, self.m = adj, np.asarray(rec), nsteps, 0
        self.inp, self.out = inp, out
        if not adj:
            for k in range(3, 9):
                self.f[k] = inp * (k - 2)
            self._sample(0)
        else:
            self._inject(nsteps)

    def _sample(self, row):
        if len(self.rec):
            k0, fz, y, x = self._taps()
            s = self.f[3]
            self.out[row] = (1 - fz) * s[k0, y, x] + fz * s[k0 + 1, y, x]

    def _inject(self, row):
        if len(self.rec):
            k0, fz, y, x = self._taps()
            for l in range(len(self.rec)):
                self.f[3, k0[l], y[l], x[l]] += (1 - fz[l]) * self.inp[row, l]
                self.f[3, k0[l] + 1, y[l], x[l]] += fz[l] * self.inp[row, l]

    def step_half(self, stress):
        if not stress:
            for i in range(3):
                self.f[i] += 0.1 * _dz_fwd(self.f[3 + i]) - 0.05 * _dz_bwd(self.f[6 + i])
        else:
            for j in range(6):
                dz = _dz_fwd if j % 2 == 0 else _dz_bwd
                self.f[3 + j] += 0.1 * dz(self.f[j % 3]) + 0.01 * j * self.f[j % 3]

    def step_receivers(self):
        self.m += 1
        if not self.adj:
            self._sample(self.m)
        else:
            self._inject(self.nsteps - self.m)
            if self.m == self.nsteps:
                self.out.copy_(self.f[3])


NSTEPS = 9


def _problem():
    rng = np.random.default_rng(7)
    p0 = torch.as_tensor(rng.standard_normal((NZ, NY, NX)))
    rec = _receivers()
    y = torch.as_tensor(rng.standard_normal((NSTEPS + 1, len(rec))))
    return p0, rec, y


def _whole():
    p0, rec, y = _problem()
    s = slabs.layout(NZ, [(0, NZ)], 0, rec)
    s.grid = FakeGrid(NZ)
    noex = lambda sl, f: None  # noqa: E731
    tr = slabs.forward([s], [p0], NSTEPS, noex)[0].clone()
    img = slabs.adjoint([s], [y], NSTEPS, noex)[0].clone()
    return tr, img


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p0, rec, y = _problem()
        parts = slabs.partition(NZ, world, NPML)
        s = slabs.layout(NZ, parts, rank, rec)
        s.grid = FakeGrid(s.nzl)
        ex = slabs.DistExchange()
        tr = slabs.forward([s], [p0[s.zl:s.zh].contiguous()], NSTEPS, ex)[0]
        img = slabs.adjoint([s], [y[:, torch.as_tensor(s.inj_idx, dtype=torch.long)].contiguous()], NSTEPS, ex)[0]
        # the whole results on every rank, and the inner products' partial sums
        full_tr = slabs.dist_gather_traces(s, tr, len(rec))
        full_img = slabs.dist_assemble_image(s, img, NZ)
        own = torch.as_tensor(s.rec_idx, dtype=torch.long)
        lhs = slabs.dist_dot(tr, y[:, own].to(tr.dtype))
        rhs = slabs.dist_dot(img[s.owned], p0[s.lo:s.hi].to(img.dtype))
        out[rank] = (s.rec_idx, tr.numpy().copy(), s.lo, s.hi, img[s.owned].numpy().copy(),
                     full_tr.numpy().copy(), full_img.numpy().copy(), lhs, rhs)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_slab_march_equals_whole_grid(world):
    tr_w, img_w = _whole()
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    L = tr_w.shape[1]
    seen = np.zeros(L, int)
    img = np.zeros((NZ, NY, NX))
    p0, _rec, y = _problem()
    lhs_w = float((tr_w.double() * y.to(tr_w.dtype).double()).sum())
    rhs_w = float((img_w.double() * p0.to(img_w.dtype).double()).sum())
    for r in range(world):
        idx, tr, lo, hi, im, full_tr, full_img, lhs, rhs = got[r]
        seen[idx] += 1
        assert np.array_equal(tr, tr_w.numpy()[:, idx])
        img[lo:hi] = im
        # every rank holds the whole traces and image, exactly
        assert np.array_equal(full_tr, tr_w.numpy())
        assert np.array_equal(full_img, img_w.numpy())
        assert abs(lhs - lhs_w) <= 1e-12 * abs(lhs_w) and abs(rhs - rhs_w) <= 1e-12 * abs(rhs_w)
    assert np.all(seen == 1)
    assert np.array_equal(img, img_w.numpy())
    assert np.abs(img).max() > 0 and np.abs(tr_w.numpy()).max() > 0
