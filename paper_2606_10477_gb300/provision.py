"""HE-DAP provisioning on this GPU (Sec. 4: run once at installation).

Runs Alg. 2 / Alg. 3 (``hedap_select``) for a parameter preset and writes the
per-level table R[l] = [u1 (accuracy), u2 (speed), u3 (absolute MRE target)]
with the full D set and per-iteration trace, keyed by device name, preset and
git revision, plus this GPU's analogue of the paper's Table 1 (Chebyshev
evaluation time per degree against the BTS time) and Table 10 (exploration
time).

  python -m paper_2606_10477_gb300.provision --preset bts16 --out provisioning.json
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import time

import numpy as np

from . import hedap, inputs


def git_revision() -> str:
    try:
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        return subprocess.run(["git", "-C", root, "rev-parse", "HEAD"], capture_output=True, text=True,
                              timeout=10).stdout.strip() or "unknown"
    except (OSError, subprocess.SubprocessError):
        return "unknown"


def device_name() -> str:
    try:
        return subprocess.run(["nvidia-smi", "--query-gpu=name", "--format=csv,noheader", "-i", "0"],
                              capture_output=True, text=True, timeout=10).stdout.strip()
    except (OSError, subprocess.SubprocessError):
        return "unknown"


def chebyshev_vs_bts(ctx, lmax, A, B_max, B, degrees, reps=3):
    """Table 1 analogue: pre-normalisation + Chebyshev evaluation at l_max, against one BTS."""
    import torch
    vals = np.linspace(A, B_max, ctx.N // 2)
    ct = ctx.encrypt(vals, lmax, 1)
    rows = []

    def timed(fn):
        best = float("inf")
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            ctx.sync()
            best = min(best, time.perf_counter() - t0)
        return 1e3 * best

    y = ctx.encrypt(vals / B_max, 1, 2)
    bts_ms = timed(lambda: ctx.bootstrap_scaled(y, 1))
    for d in degrees:
        try:
            ms = timed(lambda: ctx.invsqrt(ct, A, B_max, B, d, 0))
        except hedap.HedapError:
            continue
        rows.append({"degree": d, "cheb_ms": ms, "bts_ms": bts_ms, "ratio": ms / bts_ms})
    return rows


def parse_levels(text: str) -> list:
    """Comma-separated levels, e.g. "12,7" (empty: none)."""
    out = [int(v) for v in text.split(",") if v.strip()]
    if any(v < 0 for v in out):
        raise ValueError(f"bad level list {text!r}")
    return out


def parse_fixed(text: str) -> tuple:
    """The fixed configuration "degree,iters" (PP-STAT's is "510,6")."""
    v = tuple(int(x) for x in text.split(","))
    if len(v) != 2 or v[0] < 1 or v[1] < 0:
        raise ValueError(f"bad fixed configuration {text!r}: want degree,iters")
    return v


def parse_configs(text: str) -> list:
    """';'-separated (degree, c, iters) triples, e.g. "254,0,4;126,1,4": degree >= 1, c (Pre-BTS) 0 or 1,
    iters >= 0 (empty: none)."""
    out = []
    for e in text.split(";"):
        if not e.strip():
            continue
        v = tuple(int(x) for x in e.split(","))
        if len(v) != 3 or v[0] < 1 or v[1] not in (0, 1) or v[2] < 0:
            raise ValueError(f"bad configuration {e!r}: want degree,c,iters")
        out.append(v)
    return out


def table4(ctx, R, levels, A, B_max, B, fixed, reps=3, extra=()):
    """Table 4 analogue: at each level, CryptoInvSqrt with HE-DAP's accuracy (u1) and speed (u2) choices
    against a fixed (degree, Newton steps) configuration (PP-STAT's d = 510, i = 6 in the paper), each with
    lazy bootstrapping in the Newton loop and Pre-BTS only where the fixed degree needs it; time (CUDA
    stream synchronised, best of reps after a warm-up) and MRE against FP64 on linspace(A, B_max, N/2)."""
    import torch
    vals = np.linspace(A, B_max, ctx.N // 2)
    ref = 1 / np.sqrt(vals)
    rows = []
    for lvl in levels:
        ct = ctx.encrypt(vals, lvl, 3)
        cands = [("HE-DAP u1 (accuracy)", r["degree"], r["c"], r["iters"]) for r in R
                 if r["level"] == lvl and r["kind"] == 1]
        cands += [("HE-DAP u2 (speed)", r["degree"], r["c"], r["iters"]) for r in R
                  if r["level"] == lvl and r["kind"] == 2]
        d, i = fixed
        for c in (0, 1):
            try:
                ctx.invsqrt(ct, A, B_max, B, d, 0, c, 1 << 63)
            except hedap.HedapError:
                continue
            cands.append((f"fixed d={d}, i={i}", d, c, i))
            break
        for d, c, i in extra:  # other named configurations, where they fit the level
            try:
                ctx.invsqrt(ct, A, B_max, B, d, 0, c, 1 << 63)
            except hedap.HedapError:
                continue
            cands.append((f"given d={d}, c={c}, i={i}", d, c, i))
        for name, d, c, i in cands:
            best = float("inf")
            y = None
            for _ in range(reps + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out = ctx.invsqrt(ct, A, B_max, B, d, i, c, 1 << 63)
                ctx.sync()
                best = min(best, time.perf_counter() - t0)
                y = ctx.decrypt(out).real
            mre = float(np.mean(np.abs(y - ref) / ref))
            rows.append({"level": lvl, "config": name, "degree": d, "c": c, "iters": i, "ms": 1e3 * best,
                         "mre": mre})
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", default="bts16")
    ap.add_argument("--A", type=float, default=0.001)
    ap.add_argument("--B-max", type=float, default=100.0)
    ap.add_argument("--B", type=float, default=100.0)
    ap.add_argument("--de-min", type=int, default=4)
    ap.add_argument("--de-max", type=int, default=9)
    ap.add_argument("--i-max", type=int, default=15)
    ap.add_argument("--theta", type=float, default=1.0)
    ap.add_argument("--delta", type=float, default=1.0)
    ap.add_argument("--mre-target", type=float, default=1e-7)
    ap.add_argument("--out", default="provisioning.json")
    ap.add_argument("--table4-levels", default="", help="comma-separated levels for the Table 4 analogue")
    ap.add_argument("--fixed", default="510,6", help="the fixed (degree, Newton steps) compared in Table 4")
    ap.add_argument("--checkpoint", default="", help="also write a checkpoint (R and the NTT shapes) here")
    ap.add_argument("--extra", default="", help="more (degree,c,iters) configurations for Table 4, ';'-separated")
    args = ap.parse_args(argv)

    p = inputs.PRESETS[args.preset]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1)
    lmax = ctx.n_q - 1
    if p["hw"]:
        b = inputs.BTS
        lmax = ctx.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    t0 = time.perf_counter()
    D, R, T = ctx.select(args.A, args.B_max, args.B, args.de_min, args.de_max, args.i_max, args.theta, args.delta,
                         args.mre_target)
    explore_s = time.perf_counter() - t0
    table1 = chebyshev_vs_bts(ctx, lmax, args.A, args.B_max, args.B,
                              [(1 << e) - 2 for e in range(args.de_min, args.de_max + 1)]) if p["hw"] else []
    levels4 = parse_levels(args.table4_levels)
    fixed = parse_fixed(args.fixed)
    extra = parse_configs(args.extra)
    t4 = table4(ctx, R, levels4, args.A, args.B_max, args.B, fixed, extra=extra) if levels4 else []
    out = {
        "key": {"device": device_name(), "preset": args.preset, "params": p, "git": git_revision()},
        "config": vars(args), "l_max": lmax, "exploration_s": explore_s,
        "R": R, "D": D, "trace": T, "table1": table1, "table4": t4,
    }
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    if args.checkpoint:
        from . import checkpoint
        checkpoint.save(args.checkpoint, ctx, p, R)
    print(json.dumps({"exploration_s": explore_s, "levels": sorted({r["level"] for r in R}),
                      "R": [(r["level"], r["kind"], r["degree"], r["c"], r["iters"], r["mre"], round(r["ms"], 2))
                            for r in R], "table1": table1, "table4": t4}))


if __name__ == "__main__":
    main()
