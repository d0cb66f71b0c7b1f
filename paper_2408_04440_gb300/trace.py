"""Trace one mixed-precision factor: the per-task trace of the dataflow FP64
POTRF (``emu_trace_*``) and the per-stream timeline of the kernel groups
(``emu_prof_timeline``).

    python -m paper_2408_04440_gb300.trace [--L 128] [--nb 512] [--beta 8] [--eps 1e-8]

Prints a short text summary; ``--save PREFIX`` also writes the raw arrays as
``PREFIX_tasks.npy`` and ``PREFIX_timeline.npy``.

Records: one per worker task (TRSM, UPD), one per step of the chain (``LT``:
the 16-column step run by the master CTA, from its start to its end; "work" is
the part after its leaf) and, when the chain runs on a cluster of three
CTAs, one per step of each helper (``HELP``: block (s+1, s) and the next
diagonal block; ``HELP2``: block (s+2, s); from the inputs' arrival to the
end).
Tracing adds global stores inside the kernel, which the publishing fences then
wait for, so traced times run longer than untraced ones.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import PROF_GROUPS, Context, emu_cov_build, emu_potrf_mp

KINDS = ("LT", "TRSM", "UPD", "", "", "HELP", "HELP2")
STREAMS = ("ctx", "crit", "panel", "bulk")


def summarize_tasks(tr: np.ndarray, ntiles: int) -> list[str]:
    out = []
    if len(tr) == 0:
        return out
    per = len(tr) // ntiles
    for k in sorted({0, ntiles // 2, ntiles - 1}):
        t = tr[k * per:(k + 1) * per].astype(np.int64)
        t = t[t[:, 4] > 0]  # records that were written (the master task itself has none)
        if len(t) == 0:
            continue
        kind = t[:, 0] & 0xFF
        t0 = t[:, 2].min()
        ready, done = t[:, 3] - t0, t[:, 4] - t0
        line = f"tile {k}: span {done.max() / 1e3:.1f} us"
        for kk, nm in enumerate(KINDS):
            m = kind == kk
            if nm and m.any():
                line += f"; {nm} n={int(m.sum())} work {((done - ready)[m]).mean() / 1e3:.2f} us"
        leaf = np.sort(done[kind == 0])
        if len(leaf) > 1:
            line += f"; LT step {np.median(np.diff(leaf)) / 1e3:.1f} us (median)"
            # the chain's packed sub-phase durations in SM cycles (cluster form:
            # the leaf, the wait for X_{s+1,s} after it, the whole step)
            w = t[kind == 0, 1]
            f1, f2, step = (w >> 8) & 0x3FFFF, (w >> 26) & 0x7FFFF, (w >> 45) & 0x7FFFF
            line += (f" [cycles: leaf {np.median(f1):.0f}, wait for X {np.median(f2):.0f},"
                     f" step {np.median(step):.0f}]")
        out.append(line)
    return out


def summarize_timeline(tl: np.ndarray) -> list[str]:
    out = []
    if len(tl) == 0:
        return out
    end = tl[:, 3].max()
    for sid, name in enumerate(STREAMS):
        m = tl[:, 1] == sid
        if not m.any():
            continue
        busy = {}
        for g, t0, t1 in tl[m][:, [0, 2, 3]]:
            busy[PROF_GROUPS[int(g)]] = busy.get(PROF_GROUPS[int(g)], 0.0) + (t1 - t0)
        parts = ", ".join(f"{k} {v:.2f}" for k, v in sorted(busy.items(), key=lambda x: -x[1]))
        out.append(f"{name:5s} busy {sum(busy.values()):.2f} of {end:.2f} ms: {parts}")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--nb", type=int, default=512)
    ap.add_argument("--beta", type=float, default=8.0)
    ap.add_argument("--eps", type=float, default=1e-8)
    ap.add_argument("--save", default=None)
    a = ap.parse_args()
    with Context(0) as ctx:
        for _ in range(2):  # warm-up
            A = emu_cov_build(ctx, a.L, a.beta, a.nb)
            emu_potrf_mp(ctx, A, eps=a.eps)
            A.free()
        A = emu_cov_build(ctx, a.L, a.beta, a.nb)
        ctx.trace_enable(True)
        ctx.prof_enable(True)
        info = emu_potrf_mp(ctx, A, eps=a.eps)
        tl = ctx.prof_timeline()
        tr = ctx.trace_read()
        ctx.prof_enable(False)
        ctx.trace_enable(False)
        A.free()
    print(f"L={a.L} n={a.L * a.L} nb={a.nb} eps={a.eps:g}: factor {info.ms:.2f} ms (profiled), tiles {info.tiles}")
    for line in summarize_tasks(tr, info.nt) + summarize_timeline(tl):
        print(line)
    if a.save:
        np.save(a.save + "_tasks.npy", tr)
        np.save(a.save + "_timeline.npy", tl)


if __name__ == "__main__":
    main()
