"""Element-by-element comparison of a GPU CSR with the CPU oracle (test helper).

Tolerances (written here, used by every parity test):
  FP64 plain : |gpu - oracle| <= 1e-12 for lo, up, sink_lo, sink_up, trunc;
               column ids bit-exact (a target whose up lies within 1e-12 of
               the cutoff may fall on either side: both sides decide it in
               FP64 but with different erfc implementations).
  FP32 sound : lo32 <= lo64, up32 >= up64, sink_lo32 <= sink_lo64,
               sink_up32 >= sink_up64, every |difference| <= 2e-6, trunc
               within 2e-6; the FP32 kept set contains the FP64 kept set and
               every extra FP32 target has up64 < cutoff <= up32 (the FP32 up
               is an upper bound, so it may pass a cutoff the FP64 value
               misses by less than its error).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

TOL64 = 1e-12
TOL32 = 2e-6


@dataclass
class Report:
    rows: int = 0
    pairs: int = 0
    extra32: int = 0
    tie64: int = 0
    max_dlo: float = 0.0
    max_dup: float = 0.0
    max_dsink: float = 0.0
    max_dtrunc: float = 0.0
    failures: list = field(default_factory=list)

    def fail(self, msg):
        if len(self.failures) < 20:
            self.failures.append(msg)

    def assert_ok(self):
        assert not self.failures, "\n".join(self.failures)


def gather_rows(csr, rows):
    """Host copies of the CSR segments of `rows` (one device gather)."""
    rp = csr.row_ptr.cpu().numpy()
    rows = np.asarray(rows, dtype=np.int64)
    starts, ends = rp[rows], rp[rows + 1]
    lens = ends - starts
    if lens.sum() > 0:
        idx = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)])
        it = torch.as_tensor(idx, device=csr.col.device)
        col = csr.col.index_select(0, it).cpu().numpy()
        lo = csr.lo.index_select(0, it).cpu().numpy().astype(np.float64)
        up = csr.up.index_select(0, it).cpu().numpy().astype(np.float64)
    else:
        col = np.zeros(0, np.int32)
        lo = up = np.zeros(0)
    off = np.concatenate([[0], np.cumsum(lens)])
    rt = torch.as_tensor(rows, device=csr.col.device)
    sl = csr.sink_lo.index_select(0, rt).cpu().numpy()
    su = csr.sink_up.index_select(0, rt).cpu().numpy()
    tr = csr.trunc.index_select(0, rt).cpu().numpy()
    fl = csr.row_flags.index_select(0, rt).cpu().numpy()
    return off, col, lo, up, sl, su, tr, fl


def compare(prob, csr, orc_csr, orc, precision: str) -> Report:
    """Compare the GPU rows orc_csr.rows with the oracle's result for them."""
    rows = orc_csr.rows
    off, col, lo, up, sl, su, tr, fl = gather_rows(csr, rows)
    rep = Report(rows=len(rows))
    cut = prob.cutoff
    for k, r in enumerate(rows):
        gc, glo, gup = col[off[k]:off[k + 1]], lo[off[k]:off[k + 1]], up[off[k]:off[k + 1]]
        oc, olo, oup = orc_csr.row(k)
        rep.pairs += len(gc)
        if fl[k] != 0:
            rep.fail(f"row {r}: row_flags {fl[k]}")
        if len(gc) > 1 and np.any(np.diff(gc) <= 0):
            rep.fail(f"row {r}: columns not strictly ascending")
        common, gi, oi = np.intersect1d(gc, oc, assume_unique=True, return_indices=True)
        only_g = np.setdiff1d(gc, oc, assume_unique=True)
        only_o = np.setdiff1d(oc, gc, assume_unique=True)
        dlo = glo[gi] - olo[oi]
        dup = gup[gi] - oup[oi]
        if len(common):
            rep.max_dlo = max(rep.max_dlo, float(np.max(np.abs(dlo))))
            rep.max_dup = max(rep.max_dup, float(np.max(np.abs(dup))))
        ds = max(abs(sl[k] - orc_csr.sink_lo[k]), abs(su[k] - orc_csr.sink_up[k]))
        rep.max_dsink = max(rep.max_dsink, float(ds))
        rep.max_dtrunc = max(rep.max_dtrunc, float(abs(tr[k] - orc_csr.trunc[k])))
        if precision == "fp64":
            if len(only_g) or len(only_o):
                dense_up = orc.row_dense(prob, r)[0]
                for t in np.concatenate([only_g, only_o]):
                    if abs(dense_up[t] - cut) > TOL64:
                        rep.fail(f"row {r}: column {t} kept on one side only (up64 {dense_up[t]})")
                    rep.tie64 += 1
            if len(common) and (np.max(np.abs(dlo)) > TOL64 or np.max(np.abs(dup)) > TOL64):
                rep.fail(f"row {r}: |dlo| {np.max(np.abs(dlo)):.3g} |dup| {np.max(np.abs(dup)):.3g}")
            if ds > TOL64:
                rep.fail(f"row {r}: sink differs by {ds:.3g}")
            if abs(tr[k] - orc_csr.trunc[k]) > TOL64:
                rep.fail(f"row {r}: trunc {tr[k]} vs {orc_csr.trunc[k]}")
        else:
            if len(only_o):
                rep.fail(f"row {r}: {len(only_o)} FP64-kept targets missing in FP32")
            if len(only_g):
                dense_up = orc.row_dense(prob, r)[0]
                gmap = dict(zip(gc.tolist(), gup.tolist()))
                for t in only_g:
                    if not (dense_up[t] < cut <= gmap[int(t)] and gmap[int(t)] - TOL32 < cut):
                        rep.fail(f"row {r}: extra FP32 target {t}: up64 {dense_up[t]} up32 {gmap[int(t)]}")
                    if gmap[int(t)] < dense_up[t]:
                        rep.fail(f"row {r}: extra target {t} not bracketed")
                rep.extra32 += len(only_g)
            if len(common):
                if np.any(dlo > 0):
                    rep.fail(f"row {r}: lo32 > lo64 by {np.max(dlo):.3g}")
                if np.any(dup < 0):
                    rep.fail(f"row {r}: up32 < up64 by {-np.min(dup):.3g}")
                if np.max(np.abs(dlo)) > TOL32 or np.max(np.abs(dup)) > TOL32:
                    rep.fail(f"row {r}: |dlo| {np.max(np.abs(dlo)):.3g} |dup| {np.max(np.abs(dup)):.3g}")
            if sl[k] > orc_csr.sink_lo[k] or su[k] < orc_csr.sink_up[k]:
                rep.fail(f"row {r}: sink not bracketed ({sl[k]}, {su[k]}) vs "
                         f"({orc_csr.sink_lo[k]}, {orc_csr.sink_up[k]})")
            if ds > TOL32:
                rep.fail(f"row {r}: sink differs by {ds:.3g}")
            if abs(tr[k] - orc_csr.trunc[k]) > TOL32:
                rep.fail(f"row {r}: trunc {tr[k]} vs {orc_csr.trunc[k]}")
            # row-sum invariants of Def. 3.1 on the FP32 values themselves
            if glo.sum() + sl[k] > 1 + 1e-9 or gup.sum() + su[k] + tr[k] < 1 - 1e-9:
                rep.fail(f"row {r}: row sums violate the invariant")
    return rep
