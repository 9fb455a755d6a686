"""Benchmark: CryptoInvSqrt ciphertexts per second at N = 2^16 on one GB300.

One step = CryptoInvSqrt (Alg. 1: Chebyshev initial value + Newton) on a batch
of 8 resident ciphertexts (N = 2^16, 32768 slots, 24 x 50-bit Q primes + 2 x
60-bit P primes, two primes per key-switching digit, scale 2^50, inputs
uniform in [1e-3, 1]) with the (degree, Newton steps) pair that the sweep of
the workload's grid (degree 7/15/31/63 x 1..4 steps, key `sweep`) finds fastest
among those whose decrypted MRE is at most 1e-7 on this GPU: degree 15, 4
steps.  `value` is the batched path (the 8 ciphertexts packed into one batch,
one launch sequence, replayed from a CUDA graph; `eager` is the same sequence
launched kernel by kernel); `plain` is the same work one ciphertext per call
sequence.  `bootstrapped` times CryptoInvSqrt with bootstrapping
inside the Newton loop (N = 2^16, log2(QP) = 1555, inputs log-uniform in
[1e-4, 1]); `serving` runs Poisson arrivals of encrypted z-score / correlation
queries through the serving loop.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain C++ implementation the GPU
path is checked against) on the host cores, for the same workload, metric and
unit.  Under torchrun each rank runs its own replica (no collective); rank 0
prints.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "InvSqrt ct/s at N=2^16 (MRE<=1e-7), batched vs plain; NTT GB/s; p99 latency"
UNIT = "ct/s"
PRESET = "n16"
LO, HI, B = 1e-3, 1.0, 1.0
MRE_TARGET = 1e-7


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=8, help="ciphertexts per step")
    # (15, 4): the fastest (degree, Newton steps) of the sweep below that meets MRE <= 1e-7 on this GPU
    ap.add_argument("--degree", type=int, default=15)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bts", action="store_true", help="skip the bootstrapped workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving workload")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-level batch workload")
    ap.add_argument("--no-dnum3", action="store_true", help="skip the three-digit key-switching variant")
    ap.add_argument("--no-sweep", action="store_true", help="skip the degree x Newton-steps sweep")
    ap.add_argument("--serve-queries", type=int, default=48, help="queries in the Poisson serving run")
    ap.add_argument("--only", choices=["ntt", "serving", "mixed", "bts", "hmult", "ops"],
                    help="time only the batched NTT (for kernel profiling) or only the serving workload")
    ap.add_argument("--ntt-limbs", type=int, default=384, help="limbs per batched NTT in --only ntt")
    ap.add_argument("--profile-region", action="store_true",
                    help="--only ntt: one forward and one inverse transform between cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off); --only hmult: one batched HMult; --only bts: one batched "
                         "bootstrap")
    return ap.parse_args()


def workload_config(args, batch):
    p = __import__("paper_2606_10477_gb300.inputs", fromlist=["PRESETS"]).PRESETS[PRESET]
    return {
        "workload": (f"CryptoInvSqrt, N=2^{p['log_n']} ({2 ** (p['log_n'] - 1)} slots), {len(p['q_bits'])}x"
                     f"{p['q_bits'][0]}-bit Q + {len(p['p_bits'])}x{p['p_bits'][0]}-bit P primes, "
                     f"{p['alpha']} primes/digit, scale 2^{p['log_scale']}, inputs U[{LO},{HI}], "
                     f"Chebyshev degree {args.degree}, {args.iters} Newton steps, input level {len(p['q_bits']) - 1}"),
        "batch_ciphertexts": batch,
        "l2": "inputs larger than L2: batch of resident ciphertexts (24 MiB each) plus the 312 MiB relinearisation key",
    }


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank, int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# The NTT is bound by the integer multiply-add pipe (there is no 64-bit multiplier): a lazy Shoup
# butterfly needs the exact high half of x * w' (seven 32 x 32 half products: the low half of x0 w'0 is
# never needed) and the low halves of x * w and qh * q (two 32 x 32 -> 64 products, two slots each, and
# four low products) = 15 multiply-pipe slots per butterfly, against 64 multiply-add lanes per SM.
NTT_MUL_SLOTS_PER_BUTTERFLY = 15
IMAD_LANES_PER_SM = 64
# DRAM bytes per transformed limb: dram__bytes_read.sum + dram__bytes_write.sum of the transform launches of one
# batched HMult with rescale at the top level (`--only hmult --batch 8 --profile-region` under ncu: 4553.6 MB for
# 2912 limb transforms, the mix of fused ModUp (with the key inner product) and ModDown-rescale transforms of the
# step), scaled to a launch group by its limbs
NTT_DRAM_BYTES_PER_LIMB = 1.564e6


def ntt_alu_roofline(n, alg_bytes, ms, groups, peaks, slots):
    """The transform class against the multiply pipe.  Work = the library's algorithmic count of 32-bit
    multiply-pipe slots of the class (15 per Shoup product by a constant: every butterfly and every product of
    a fused basis conversion; 8 per 64 x 64 -> 128-bit product of the fused key inner product); peak = SMs x 64
    multiply-add lanes x clock.  The butterfly-only view (the transforms' butterflies against 15 slots each) is
    kept beside it."""
    log_n = int(n).bit_length() - 1
    limbs = alg_bytes / (16.0 * n)
    bfly = limbs * (n // 2) * log_n
    sec = ms / 1e3 if ms > 0 else float("inf")
    mhz = peaks.get("sm_max_mhz", 2070.0)
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peak_slots = sms * IMAD_LANES_PER_SM * mhz * 1e6
    achieved = slots / sec / 1e12
    peak = peak_slots / 1e12
    bfly_peak = peak_slots / NTT_MUL_SLOTS_PER_BUTTERFLY / 1e9
    return {"kernel": "ntt", "bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "Tslot/s (32-bit multiply-pipe slots)", "frac": achieved / peak,
            "traffic": NTT_DRAM_BYTES_PER_LIMB * limbs / max(1, groups),
            "traffic_unit": "bytes per launch group (ncu, scaled per limb)",
            "algorithmic_bytes_per_group": alg_bytes / max(1, groups),
            "algorithmic_slots_per_group": slots / max(1, groups),
            "peak_source": f"derived: {sms} SMs (read from the device) x {IMAD_LANES_PER_SM} integer multiply-add "
                           f"lanes x {mhz:.0f} MHz",
            "launch_groups": groups, "avg_group_us": 1e3 * ms / max(1, groups),
            "butterfly_view": {"achieved_gbutterfly_s": bfly / sec / 1e9, "peak_gbutterfly_s": bfly_peak,
                               "frac": bfly / sec / 1e9 / bfly_peak,
                               "butterflies_per_group": bfly / max(1, groups),
                               "peak_source": f"{NTT_MUL_SLOTS_PER_BUTTERFLY} multiply slots per Shoup butterfly"}}


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_invsqrt_seconds(args, seed=1):
    """One full oracle CryptoInvSqrt on the benchmark workload; returns (seconds, threads, MRE)."""
    import oracle
    from paper_2606_10477_gb300 import inputs
    p = inputs.PRESETS[PRESET]
    ctx = oracle.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], seed)
    a = inputs.uniform_values(seed, ctx.N // 2, LO, HI)
    ct = ctx.encrypt(a, ctx.n_q - 1, seed + 100)
    t0 = time.perf_counter()
    out = ctx.invsqrt(ct, LO, HI, B, args.degree, args.iters)
    dt = time.perf_counter() - t0
    y = ctx.decrypt(out).real
    ref = 1 / np.sqrt(a)
    return dt, oracle.threads(), float(np.mean(np.abs(y - ref) / ref))


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    steps = max(1, args.steps)
    times = []
    mre = None
    for i in range(args.warmup + steps):
        dt, threads, mre = oracle_invsqrt_seconds(args, seed=1 + i)
        if i >= args.warmup:
            times.append(dt)
        if i == 0 and dt * (args.warmup + steps) > 240:  # keep the whole run within a few minutes
            args.warmup, steps = 0, 1
            times = [dt]
            break
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(args, 1),
        "mre": mre,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "one full oracle CryptoInvSqrt of one ciphertext per step (same parameters)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU path
def run_ours(args):
    import torch
    from paper_2606_10477_gb300 import hedap, inputs, replicas
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    p = inputs.PRESETS[PRESET]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"],
                        replicas.rank_seed(1, rank), stream=stream.cuda_stream)
    L = ctx.n_q - 1
    batch = args.batch
    vals = [inputs.uniform_values(1000 * rank + i, ctx.N // 2, LO, HI) for i in range(batch)]
    cts = [ctx.encrypt(v, L, 7 + i) for i, v in enumerate(vals)]

    packed = ctx.pack(cts)

    def step():  # batched: the whole batch through one launch sequence
        return ctx.invsqrt(packed, LO, HI, B, args.degree, args.iters)

    def step_plain():  # one ciphertext per call sequence
        return [ctx.invsqrt(c, LO, HI, B, args.degree, args.iters) for c in cts]

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # accuracy of this configuration on the batch (untimed)
    out_b = step()
    mres = []
    for k, v in enumerate(vals):
        y = ctx.decrypt(ctx.unpack(out_b, k)).real
        ref = 1 / np.sqrt(v)
        mres.append(float(np.mean(np.abs(y - ref) / ref)))
    out_level = out_b.level
    del out_b
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps on resident inputs, each one replay of the batched step captured
    # as a CUDA graph (the same launch sequence as step(), bit for bit)
    graph_b = ctx.invsqrt_graph(packed, LO, HI, B, args.degree, args.iters)
    for _ in range(args.warmup):
        graph_b.run(want_output=False)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph_b.run(want_output=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    elapsed_ms = e0.elapsed_time(e1)
    launches = graph_b.kernels * args.steps
    clk = clocks.stop()
    value, tmax_s, _ = replicas.aggregate(batch * args.steps, elapsed_ms / 1e3,
                                          torch.distributed if ws > 1 else None)
    elapsed_ms = tmax_s * 1e3
    graph_kernels = graph_b.kernels
    graph_b.close()

    # ---- the same batched step launched kernel by kernel (no graph)
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = hedap.launch_count()
    t0e.record(stream)
    for _ in range(args.steps):
        step()
    t1e.record(stream)
    torch.cuda.synchronize()
    eager_value = batch * args.steps / (t0e.elapsed_time(t1e) / 1e3)
    eager_launches = (hedap.launch_count() - launches0) / args.steps

    # ---- the plain path, same work and timing
    step_plain()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(max(1, min(args.steps, 3))):
        step_plain()
    p1.record(stream)
    torch.cuda.synchronize()
    plain_value = batch * max(1, min(args.steps, 3)) / (p0.elapsed_time(p1) / 1e3)

    # ---- one ciphertext per replay of a graph captured for a single ciphertext
    graph_1 = ctx.invsqrt_graph(cts[0], LO, HI, B, args.degree, args.iters)
    for _ in range(2):
        graph_1.run(cts[0], want_output=False)
    torch.cuda.synchronize()
    g_lat = []
    for c in cts:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        graph_1.run(c, want_output=False)
        b.record(stream)
        b.synchronize()
        g_lat.append(a.elapsed_time(b))
    graph_info = {"plain_ms_p50": float(np.percentile(g_lat, 50)), "plain_value": 1e3 / float(np.mean(g_lat)),
                  "unit": UNIT, "kernels_per_replay_batched": graph_kernels,
                  "kernels_per_replay_plain": graph_1.kernels}
    graph_1.close()

    # ---- per-ciphertext latency (plain path: one ciphertext per call sequence)
    lat = []
    for c in cts:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.invsqrt(c, LO, HI, B, args.degree, args.iters)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))

    # ---- same steps with the per-kernel-class event profiler on
    hedap.profile_enable(True)
    n_prof_steps = max(1, min(args.steps, 2))
    for _ in range(n_prof_steps):
        step()
    torch.cuda.synchronize()
    prof = hedap.profile_read()
    ntt_slots = hedap.profile_read_slots("ntt")
    hedap.profile_enable(False)
    total_prof_ms = sum(v[1] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][1])
    n_dom, ms_dom, by_dom = prof[dom]
    peaks, peak_kind = measured_peaks()
    achieved = by_dom / (ms_dom / 1e3) / 1e9 if ms_dom > 0 else 0.0
    ntt = prof["ntt"]
    ntt_gbs = ntt[2] / (ntt[1] / 1e3) / 1e9 if ntt[1] > 0 else None
    if dom == "ntt":
        # the transforms are bound by the integer multiply-add pipe, not HBM: their algorithmic multiply work
        # (butterflies, fused conversions and inner-product products) against that pipe's slot rate
        roofline = ntt_alu_roofline(ctx.N, by_dom, ms_dom, n_dom, peaks, ntt_slots)
        roofline["butterfly_view"]["register_loop_gbutterfly_s"] = ctx.butterfly_rate() / 1e9
    else:
        roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_kind,
                    "launch_groups": n_dom, "avg_group_us": 1e3 * ms_dom / max(1, n_dom)}
    roofline["hbm_view"] = {"achieved_gbs": achieved, "peak_gbs": peaks["hbm_gbs"],
                            "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_kind}
    # the HBM-bound kernel classes of the same step, against measured HBM (algorithmic bytes: each input word
    # read once, each output word written once, per launch group)
    hbm_kernels = []
    for cls in ("tensor", "elementwise", "ksk_inner", "automorph", "rescale", "moddown", "modup"):
        n_c, ms_c, by_c = prof[cls]
        if n_c and ms_c > 0:
            a_c = by_c / (ms_c / 1e3) / 1e9
            hbm_kernels.append({"kernel": cls, "bound": "hbm", "achieved": a_c, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                "frac": a_c / peaks["hbm_gbs"], "traffic": None, "peak_source": peak_kind,
                                "launch_groups_per_step": n_c / n_prof_steps, "avg_group_us": 1e3 * ms_c / n_c})

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region
    host_in = torch.empty((batch, 2, L + 1, ctx.N), dtype=torch.int64, pin_memory=True)
    for k, c in enumerate(cts):
        host_in[k].numpy()[...] = c.limbs().view(np.int64)
    host_out = torch.empty((batch, 2, out_level + 1, ctx.N), dtype=torch.int64, pin_memory=True)
    h2d = host_in.numel() * 8
    d2h = host_out.numel() * 8

    graph_e = ctx.invsqrt_graph(packed, LO, HI, B, args.degree, args.iters)

    def e2e_step():  # the batch's host limbs in (one copy), the captured step, the batch's host limbs out (one copy)
        out = graph_e.run(ctx.batch_import(host_in, batch, L, ctx.scale))
        ctx.batch_export(out, host_out)

    e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    k_e2e = max(1, min(args.steps, 10))
    for _ in range(k_e2e):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value, e2e_s, _ = replicas.aggregate(batch * k_e2e, e2e_s, torch.distributed if ws > 1 else None)
    graph_e.close()

    # ---- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        dt, threads, omre = oracle_invsqrt_seconds(args)
        cpu = {"value": 1.0 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "one full oracle CryptoInvSqrt of one ciphertext on the same workload", "mre": omre}

    ntt = measure_ntt(ctx, inputs, torch, stream, 384)
    ops = per_op_us(ctx, inputs, torch, stream, batch)
    sweep = None if args.no_sweep else config2_sweep(ctx, hedap, inputs, torch, stream, packed, vals)
    bts = None if args.no_bts else bootstrapped_workload(ctx_cls=hedap.Context, inputs=inputs, torch=torch,
                                                         stream=stream, rank=rank, batch=batch)
    mixed = None if args.no_mixed else mixed_workload(hedap, inputs, torch, stream, rank)
    dnum3 = None if args.no_dnum3 else dnum3_variant(hedap, inputs, torch, stream, rank, batch, args.degree,
                                                     args.iters, args.steps)
    serving = None if args.no_serving else serving_workload(hedap, inputs, torch, stream, rank, args.serve_queries)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args, batch),
            "mre": max(mres), "mre_target": MRE_TARGET,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "ntt_gbs": ntt_gbs,
            "ntt_batched": ntt,
            "ntt_shapes": ctx.ntt_get_roles(),
            "per_op_us": ops,
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "roofline": roofline,
            "roofline_hbm_kernels": hbm_kernels,
            "profile_share": {k: round(v[1] / total_prof_ms, 4) for k, v in prof.items()} if total_prof_ms else {},
            "profile_classes": {k: {"groups_per_step": v[0] / n_prof_steps, "ms_per_step": v[1] / n_prof_steps,
                                    "us_per_group": 1e3 * v[1] / v[0], "algorithmic_gbs": v[2] / (v[1] / 1e3) / 1e9}
                                for k, v in prof.items() if v[0] > 0},
            "cpu_baseline": cpu,
            "execution": "each timed step is one replay of the batched InvSqrt launch sequence captured as a "
                         "CUDA graph (hedap_graph_run); eager = the same sequence launched kernel by kernel",
            "eager": {"value": eager_value, "unit": UNIT, "kernels_per_step": eager_launches},
            "plain": {"value": plain_value, "unit": UNIT, "ms_per_ct": 1e3 / plain_value,
                      "speedup_batched_vs_plain": value / plain_value},
            "graph": graph_info,
            "bootstrapped": bts,
            "dnum3_variant": dnum3,
            "sweep": sweep,
            "mixed_levels": mixed,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def bootstrapped_workload(ctx_cls, inputs, torch, stream, rank, batch, steps=2):
    """CryptoInvSqrt with lazy bootstrapping in the Newton loop: N = 2^16, bts16 chain
    (log2 QP = 1555, h = 192), inputs log-uniform in [1e-4, 1] at l_max, batch of ciphertexts, with
    (d, c, i) chosen by HE-DAP's selector (Alg. 2 / Alg. 3) on this GPU for MRE <= 1e-7 at l_max."""
    p = inputs.PRESETS["bts16"]
    b = inputs.BTS
    t0 = time.perf_counter()
    ctx = ctx_cls(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 11 + rank,
                  stream=stream.cuda_stream)
    lmax = ctx.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    lo = 1e-4
    s0 = time.perf_counter()
    _, R, _ = ctx.select(lo, 1.0, 1.0, 4, 7, 8, mre_target=1e-7, level_min=lmax, level_max=lmax)
    choice = next((r for r in R if r["kind"] == 3), None) or next(r for r in R if r["kind"] == 1)
    degree, iters, pre = choice["degree"], choice["iters"], choice["c"]
    select_s = time.perf_counter() - s0
    vals = [inputs.log_uniform_values(2000 + i, ctx.N // 2, lo, 1.0) for i in range(batch)]
    packed = ctx.pack([ctx.encrypt(v, lmax, 3000 + i) for i, v in enumerate(vals)])
    mask = 1 << 63
    out = ctx.invsqrt(packed, lo, 1.0, 1.0, degree, iters, pre, mask)  # warm-up: keys and diagonals are built here
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    mres = []
    for k, v in enumerate(vals):
        y = ctx.decrypt(ctx.unpack(out, k)).real
        mres.append(float(np.mean(np.abs(y - 1 / np.sqrt(v)) * np.sqrt(v))))
    # eager: the batched step launched kernel by kernel
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(2):
        ctx.invsqrt(packed, lo, 1.0, 1.0, degree, iters, pre, mask)
    e1.record(stream)
    torch.cuda.synchronize()
    eager_ms = e0.elapsed_time(e1) / 2
    # timed: the batched step captured as a CUDA graph and replayed for at least a second (inputs resident
    # and larger than L2), clocks sampled during the replays
    graph = ctx.invsqrt_graph(packed, lo, 1.0, 1.0, degree, iters, pre, mask)
    graph.run(want_output=False)
    torch.cuda.synchronize()
    steps = max(steps, int(np.ceil(1000.0 / max(eager_ms, 1.0))) + 1)
    clk = ClockSampler()
    e0.record(stream)
    for _ in range(steps):
        graph.run(want_output=False)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / steps
    graph.close()
    single = ctx.encrypt(vals[0], lmax, 4000)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    ctx.invsqrt(single, lo, 1.0, 1.0, degree, iters, pre, mask)
    s1.record(stream)
    torch.cuda.synchronize()
    bts_ct = ctx.encrypt(vals[0] / 2, 1, 5000)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    ctx.bootstrap_scaled(bts_ct, 1)
    b1.record(stream)
    torch.cuda.synchronize()
    bootstrap_ms = b0.elapsed_time(b1)
    sparse = {}
    for ls in (10, 13):  # sparse packing: 2^ls values repeated over the N/2 slots
        n = 1 << ls
        v = inputs.uniform_values(5100 + ls, n, -1, 1) + 1j * inputs.uniform_values(5200 + ls, n, -1, 1)
        zt = np.tile(v, ctx.N // 2 // n)
        sct = ctx.encrypt(zt, 1, 5300 + ls)
        err = np.abs(ctx.decrypt(ctx.bootstrap_scaled_slots(sct, 1, ls)) - zt)  # warm-up builds its diagonals
        torch.cuda.synchronize()
        b0.record(stream)
        ctx.bootstrap_scaled_slots(sct, 1, ls)
        b1.record(stream)
        torch.cuda.synchronize()
        sparse[f"2^{ls}"] = {"bootstrap_ms": b0.elapsed_time(b1), "max_err": float(err.max()),
                             "mean_err": float(err.mean())}
    ctx.close()
    dense = dense_secret_bootstrap(ctx_cls, inputs, torch, stream, rank)
    return {"workload": f"CryptoInvSqrt with lazy bootstrapping, N=2^16, log2(QP)=1555, h=192, inputs log-U[{lo},1] "
                        f"at level {lmax}, (degree {degree}, Pre-BTS {pre}, {iters} Newton steps) chosen by the "
                        f"selector for MRE <= 1e-7, batch {batch}",
            "selected": choice, "select_s": select_s,
            "value": batch * 1e3 / ms, "unit": UNIT, "ms_per_batch": ms, "mre": max(mres),
            "execution": f"batched step captured as a CUDA graph, {steps} replays timed with CUDA events "
                         f"({steps * ms / 1e3:.2f} s)", "steps": steps, "clocks": clocks,
            "eager_value": batch * 1e3 / eager_ms, "plain_value": 1e3 / s0.elapsed_time(s1),
            "speedup_batched_vs_plain": (batch * 1e3 / ms) / (1e3 / s0.elapsed_time(s1)),
            "plain_ms_per_ct": s0.elapsed_time(s1), "bootstrap_ms": bootstrap_ms, "setup_s": setup_s,
            "bootstrap_sparse_slots": sparse, "bootstrap_dense_secret": dense}


def dense_secret_bootstrap(ctx_cls, inputs, torch, stream, rank, steps=3):
    """One bootstrap under a dense ternary secret through sparse-secret encapsulation (an ephemeral
    weight-192 secret; two key switches more than the sparse chain), N = 2^16, bts16d chain: time and
    decrypted error of 32768 complex slots in [-1, 1]."""
    p = inputs.PRESETS["bts16d"]
    b = inputs.BTS
    ctx = ctx_cls(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 61 + rank,
                  stream=stream.cuda_stream)
    ctx.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    ctx.bts_encapsulate(inputs.ENC_HW)
    half = ctx.N // 2
    z = inputs.uniform_values(8000, half, -1, 1) + 1j * inputs.uniform_values(8001, half, -1, 1)
    ct = ctx.encrypt(z, 1, 8002)
    out = ctx.bootstrap_scaled(ct, 1)  # warm-up: keys and diagonals are built here
    err = np.abs(ctx.decrypt(out) - z)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.bootstrap_scaled(ct, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    return {"workload": "bootstrapping under a dense ternary secret with sparse-secret encapsulation (h = 192), "
                        "N=2^16, log2(QP)=1605, 32768 complex slots",
            "bootstrap_ms": e0.elapsed_time(e1) / steps, "max_err": float(err.max()), "mean_err": float(err.mean())}


def dnum3_variant(hedap, inputs, torch, stream, rank, batch, degree, iters, steps):
    """The same InvSqrt step on the same ring with three key-switching digits (dnum = 3, as the
    workload names it; 7 special primes of 60 bits instead of 2 so that P exceeds a 400-bit digit)."""
    p = inputs.PRESETS["n16d3"]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 51 + rank,
                        stream=stream.cuda_stream)
    L = ctx.n_q - 1
    vals = [inputs.uniform_values(7000 + i, ctx.N // 2, LO, HI) for i in range(batch)]
    packed = ctx.pack([ctx.encrypt(v, L, 7100 + i) for i, v in enumerate(vals)])
    out = ctx.invsqrt(packed, LO, HI, B, degree, iters)
    mres = []
    for k, v in enumerate(vals):
        y = ctx.decrypt(ctx.unpack(out, k)).real
        mres.append(float(np.mean(np.abs(y * np.sqrt(v) - 1))))
    graph = ctx.invsqrt_graph(packed, LO, HI, B, degree, iters)
    for _ in range(2):
        graph.run(want_output=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        graph.run(want_output=False)
    e1.record(stream)
    torch.cuda.synchronize()
    value = batch * steps / (e0.elapsed_time(e1) / 1e3)
    graph.close()
    ctx.close()
    return {"workload": f"as the main step with 8 primes per key-switching digit (dnum 3) and 7 x 60-bit special "
                        f"primes, batch {batch}", "value": value, "unit": UNIT, "mre": max(mres)}


def mixed_workload(hedap, inputs, torch, stream, rank, n_cts=64):
    """The batched workload: 64 ciphertexts at N=2^16 at mixed levels and slot counts on the FGb-shaped
    bootstrapping chain (bts16f, 12 levels after bootstrapping): limbs ~ U{3..13} (levels 2..12, every
    level a user ciphertext can have on this chain), 2^U{10..15} slots (the values repeated to fill N/2
    slots), inputs log-uniform in [1e-4, 1].  Each member's (degree, Pre-BTS, Newton steps) is HE-DAP's
    choice at its level (Alg. 3 on this GPU: u3, the fastest with MRE <= 1e-7, else u1), with lazy
    bootstrapping.  Executions of the same work: one ciphertext per call (sparse-slot bootstraps),
    hedap_invsqrt_mixed with per-member slot counts, hedap_invsqrt_mixed with full-slot bootstraps for every
    member (valid for any packing; larger batches), and the latter captured as one CUDA graph."""
    p = inputs.PRESETS["bts16f"]
    b = inputs.BTS
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 31 + rank,
                        stream=stream.cuda_stream)
    lmax = ctx.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    lo = 1e-4
    s0 = time.perf_counter()
    _, R, _ = ctx.select(lo, 1.0, 1.0, 4, 5, 8, mre_target=1e-7)
    select_s = time.perf_counter() - s0
    table = {}
    for r in R:
        if r["kind"] in (1, 3) and (r["level"] not in table or r["kind"] == 3):
            table[r["level"]] = r
    rng = np.random.default_rng(41 + rank)
    levels = rng.integers(2, lmax + 1, n_cts)
    log_slots = rng.integers(10, 16, n_cts)
    half = ctx.N // 2
    vals = [inputs.log_uniform_values(5000 + i, 1 << int(s), lo, 1.0) for i, s in enumerate(log_slots)]
    cts = [ctx.encrypt(np.tile(v, half // v.size), int(l), 6000 + i) for i, (v, l) in enumerate(zip(vals, levels))]
    mask = 1 << 63

    def cfg(i, slot_aware):
        e = table[int(levels[i])]
        ls = int(log_slots[i]) if slot_aware and int(log_slots[i]) < ctx.log_n - 1 else 0
        return (lo, 1.0, 1.0, e["degree"], e["iters"], e["c"], mask, ls)

    sparse_cfgs = [cfg(i, True) for i in range(n_cts)]
    full_cfgs = [cfg(i, False) for i in range(n_cts)]

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    def mre(outs):
        worst = 0.0
        for v, o in zip(vals, outs):
            y = ctx.decrypt(o).real[:v.size]
            worst = max(worst, float(np.mean(np.abs(y * np.sqrt(v) - 1))))
        return worst

    res = {}
    ctx.invsqrt_mixed(cts, sparse_cfgs)  # warm-up: every level's constants and both kinds of diagonals
    ctx.invsqrt_mixed(cts, full_cfgs)
    for name, fn in (("plain", lambda: [ctx.invsqrt(c, *f) for c, f in zip(cts, sparse_cfgs)]),
                     ("mixed_per_member_slots", lambda: ctx.invsqrt_mixed(cts, sparse_cfgs)),
                     ("mixed_full_slot_bootstraps", lambda: ctx.invsqrt_mixed(cts, full_cfgs))):
        outs, sec = timed(fn)
        res[name] = {"value": n_cts / sec, "unit": UNIT, "seconds": sec, "max_mre": mre(outs)}
    graph = ctx.invsqrt_mixed_graph(cts, full_cfgs)
    graph.run_many(want_output=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    e0.record(stream)
    for _ in range(reps):
        graph.run_many(want_output=False)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3 / reps
    outs = graph.run_many(cts)
    res["graph_full_slot_bootstraps"] = {"value": n_cts / sec, "unit": UNIT, "seconds": sec, "max_mre": mre(outs),
                                         "kernels_per_replay": graph.kernels}
    graph.close()
    ctx.close()
    res["workload"] = (f"{n_cts} ciphertexts, N=2^16 FGb-shaped chain (log2 QP 1545, l_max {lmax}), levels "
                       f"U{{2..{lmax}}}, slots 2^U{{10..15}}, inputs log-U[1e-4,1], per-level (d, c, i) from HE-DAP's "
                       f"table on this GPU, lazy bootstrapping")
    res["table"] = {int(k): (v["degree"], v["c"], v["iters"], v["kind"]) for k, v in sorted(table.items())}
    res["select_s"] = select_s
    res["speedup_mixed_vs_plain"] = res["mixed_full_slot_bootstraps"]["value"] / res["plain"]["value"]
    res["speedup_graph_vs_plain"] = res["graph_full_slot_bootstraps"]["value"] / res["plain"]["value"]
    return res


def config2_sweep(ctx, hedap, inputs, torch, stream, packed, vals, degrees=(7, 15, 31, 63), iters=(1, 2, 3, 4)):
    """The N=2^16 workload's sweep: Chebyshev degree d x Newton steps k on the same resident batch, each
    point with its decrypted MRE (worst member), output level, batched device time per step (CUDA events,
    best of 3 after a warm-up) and its per-kernel-class device time (event profiler, one run)."""
    rows = []
    for d in degrees:
        for k in iters:
            out = ctx.invsqrt(packed, LO, HI, B, d, k)
            worst = 0.0
            for m, v in enumerate(vals):
                y = ctx.decrypt(ctx.unpack(out, m)).real
                worst = max(worst, float(np.mean(np.abs(y * np.sqrt(v) - 1))))
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.invsqrt(packed, LO, HI, B, d, k)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            hedap.profile_enable(True)
            ctx.invsqrt(packed, LO, HI, B, d, k)
            torch.cuda.synchronize()
            prof = hedap.profile_read()
            hedap.profile_enable(False)
            rows.append({"degree": d, "newton_iters": k, "mre": worst, "meets_target": worst <= MRE_TARGET,
                         "output_level": out.level, "ms_per_batch": best, "ct_per_s": packed.batch * 1e3 / best,
                         "class_ms": {c: round(v[1], 3) for c, v in prof.items() if v[0] > 0}})
    ok = [r for r in rows if r["meets_target"]]
    fastest = max(ok, key=lambda r: r["ct_per_s"]) if ok else None
    return {"batch": packed.batch, "rows": rows,
            "fastest_meeting_target": {"degree": fastest["degree"], "newton_iters": fastest["newton_iters"],
                                       "ct_per_s": fastest["ct_per_s"], "mre": fastest["mre"]} if fastest else None}


SERVE_RECORDS = [1 << 10, 1 << 12, 1 << 14, 1 << 16, 1 << 18, 1 << 20]
SERVE_ZCFG = (1e-3, 1.0, 1.0, 31, 4, 0, 1 << 63)  # variance of the records (sd 0.1): [1e-3, 1]
SERVE_PCFG = (1e-5, 1e-2, 1e-2, 31, 5, 0, 1 << 63)  # product of two variances: [1e-5, 1e-2]


def serving_workload(hedap, inputs, torch, stream, rank, n_queries, max_batch=8):
    """Poisson arrivals of encrypted z-score / correlation queries (half each) over 2^10..2^20
    Gaussian records (mean 50, sd 10, in units of 100) packed into N=2^16 ciphertexts at the
    bootstrapped level; InvSqrt of the variance with lazy bootstrapping; keys resident."""
    p = inputs.PRESETS["bts16"]
    b = inputs.BTS
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 21 + rank,
                        stream=stream.cuda_stream)
    lvl = ctx.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"]) + 3  # 3 levels above a bootstrapped one
    slots = ctx.N // 2
    pool = []
    rhos = np.random.default_rng(77 + rank).uniform(-0.9, 0.9, len(SERVE_RECORDS))
    for k, n in enumerate(SERVE_RECORDS):
        x = inputs.gaussian_records(500 + k, n)
        y = inputs.correlated_records(600 + k, x, float(rhos[k]))
        gx = [ctx.encrypt(v, lvl, 7000 + 100 * k + i) for i, v in enumerate(inputs.pack_slots(x, slots))]
        gy = [ctx.encrypt(v, lvl, 8000 + 100 * k + i) for i, v in enumerate(inputs.pack_slots(y, slots))]
        pool.append((n, x, y, gx, gy))
    rng = np.random.default_rng(99 + rank)

    def submit(srv, kind, k):
        n, _, _, gx, gy = pool[k]
        if kind == hedap.QUERY_ZSCORE:
            return srv.submit(kind, gx, n, SERVE_ZCFG)
        return srv.submit(kind, gx, n, SERVE_PCFG, ys=gy)

    def plan(m):
        return [(hedap.QUERY_ZSCORE if i % 2 == 0 else hedap.QUERY_PCC, int(rng.integers(len(pool))))
                for i in range(m)]

    # warm-up (bootstrapping diagonals, key-switching buffers) and accuracy of one query of each kind
    srv = hedap.Server(ctx, max_batch=max_batch)
    kz, kp = len(pool) - 1, 3
    _, zs, _ = srv.poll(submit(srv, hedap.QUERY_ZSCORE, kz))
    _, rs, _ = srv.poll(submit(srv, hedap.QUERY_PCC, kp))
    n, x, _, _, _ = pool[kz]
    z = np.concatenate([ctx.decrypt(c).real for c in zs])[:n]
    z_err = float(np.max(np.abs(z - (x - x.mean()) / x.std())))
    n, x, y, _, _ = pool[kp]
    r_err = float(np.max(np.abs(ctx.decrypt(rs[0]).real - np.corrcoef(x, y)[0, 1])))
    srv.close()

    # capacity: a burst released at once
    burst = plan(2 * max_batch)
    srv = hedap.Server(ctx, max_batch=max_batch, paused=True)
    ids = [submit(srv, kind, k) for kind, k in burst]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    srv.resume()
    for i in ids:
        srv.poll(i)
    capacity = len(ids) / (time.perf_counter() - t0)
    srv.close()

    # Poisson arrivals at fractions of that capacity
    def poisson(frac, m):
        rate = frac * capacity
        arrivals = np.cumsum(rng.exponential(1.0 / rate, m))
        queries = plan(m)
        srv = hedap.Server(ctx, max_batch=max_batch)
        t0 = time.perf_counter()
        ids = []
        for (kind, k), t in zip(queries, arrivals):
            wait = t0 + t - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            ids.append(submit(srv, kind, k))
        groups = [srv.poll(i)[2]["group_size"] for i in ids]
        st = srv.stats()
        merged = srv.merges()
        srv.close()
        records = sum(pool[k][0] for _, k in queries)
        return {"load": frac, "arrival_rate_qps": rate, "queries": m, "qps": st["qps"], "p50_ms": st["p50_ms"],
                "p99_ms": st["p99_ms"], "records_per_s": records * st["qps"] / m,
                "mean_group_size": float(np.mean(groups)), "merged_groups": merged}

    main = poisson(0.75, n_queries)
    sweep = [poisson(f, n_queries) for f in (0.25, 0.5, 0.9)]
    ctx.close()
    return {"workload": f"Poisson arrivals, {n_queries} queries (z-score / PCC alternating) over "
                        f"{SERVE_RECORDS[0]}..{SERVE_RECORDS[-1]} Gaussian records (mean 50, sd 10, /100; PCC pairs "
                        f"with rho ~ U[-0.9, 0.9]), N=2^16 bts16 chain, inputs at level {lvl} (3 above a bootstrapped "
                        f"ciphertext), InvSqrt degree 31 with lazy bootstrapping, max_batch {max_batch}, "
                        f"arrival rate 0.75 x burst capacity",
            "qps": main["qps"], "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"],
            "arrival_rate_qps": main["arrival_rate_qps"], "burst_capacity_qps": capacity,
            "records_per_s": main["records_per_s"], "mean_group_size": main["mean_group_size"],
            "load_sweep": sweep, "zscore_max_abs_err": z_err, "pcc_abs_err": r_err}


def run_serving_only(args):
    import torch
    from paper_2606_10477_gb300 import hedap, inputs
    stream = torch.cuda.current_stream()
    r = serving_workload(hedap, inputs, torch, stream, 0, args.serve_queries)
    print(json.dumps({"metric": "queries/s (serving, Poisson arrivals)", "value": r["qps"], "unit": "queries/s",
                      "higher_is_better": True, "serving": r}), flush=True)


def measure_ntt(ctx, inputs, torch, stream, limbs, reps=5, profile_region=False):
    """Batched forward and inverse NTT over `limbs` limbs of N = 2^16 words resident in HBM
    (polynomials of n_q limbs, one launch per phase): algorithmic GB/s = limbs * N * 16 B
    (each word read and written once) per transform."""
    primes = ctx.primes()[:ctx.n_q]
    polys = max(1, limbs // len(primes))
    host = np.concatenate([inputs.random_limbs(9000 + i, primes, ctx.N) for i in range(polys)])
    buf = torch.from_numpy(host.view(np.int64)).cuda()
    limbs = polys * len(primes)

    def run(inverse):
        ctx.ntt_batch(buf, len(primes), 0, inverse=inverse)

    run(False)
    run(True)
    torch.cuda.synchronize()
    assert np.array_equal(buf.cpu().numpy().view(np.uint64), host), "NTT round trip failed"
    out = {}
    for name, inv in (("forward", False), ("inverse", True)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run(inv)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        bfly = limbs * (ctx.N // 2) * (ctx.N.bit_length() - 1)
        out[name] = {"ms": ms, "gbs": limbs * ctx.N * 16 / (ms / 1e3) / 1e9, "us_per_limb": 1e3 * ms / limbs,
                     "gbutterfly_s": bfly / (ms / 1e3) / 1e9}
    out["limbs"] = limbs
    if profile_region:  # one forward and one inverse transform inside a profiler capture region
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        run(False)
        run(True)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    return out


def per_op_us(ctx, inputs, torch, stream, batch, reps=10):
    """Device time of single operations at the top level of the N=2^16 workload chain, one ciphertext
    and a batch of `batch` (CUDA events over `reps` calls each, after one untimed call)."""
    L = ctx.n_q - 1
    out = {}
    for b in (1, batch):
        cts = [ctx.encrypt(inputs.uniform_values(9700 + i, ctx.N // 2, LO, HI), L, 9800 + i) for i in range(b)]
        x = ctx.pack(cts) if b > 1 else cts[0]
        r = ctx.mul_relin(x, x)
        ops = {
            "hmult (tensor, key switch, rescale)": lambda: ctx.mul(x, x),
            "tensor + key switch": lambda: ctx.mul_relin(x, x),
            "rescale": lambda: ctx.rescale(r),
            "rotation by 1": lambda: ctx.rotate(x, 1),
            "conjugation": lambda: ctx.conjugate(x),
            "constant multiply + rescale": lambda: ctx.mul_const(x, 1.5, x.scale),
            "addition": lambda: ctx.add(x, x),
        }
        row = {}
        for name, fn in ops.items():
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            row[name] = 1e3 * e0.elapsed_time(e1) / reps
        out[f"batch {b}"] = row
    out["level"] = L
    return out


def run_ops_only(args):
    import torch
    from paper_2606_10477_gb300 import hedap, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    p = inputs.PRESETS[PRESET]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1,
                        stream=stream.cuda_stream)
    print(json.dumps({"per_op_us": per_op_us(ctx, inputs, torch, stream, args.batch)}), flush=True)


def run_hmult_only(args):
    """One batched HMult (tensor, key switch with the fused ModUp / ModDown transforms, rescale) of
    `--batch` ciphertexts at the top level of the N=2^16 workload chain: its time and the NTT class's
    algorithmic bytes (limbs transformed x N x 16 B) from the event profiler, the unit the DRAM
    traffic of its NTT launches is scaled by."""
    import torch
    from paper_2606_10477_gb300 import hedap, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    p = inputs.PRESETS[PRESET]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1,
                        stream=stream.cuda_stream)
    L = ctx.n_q - 1
    vals = [inputs.uniform_values(9500 + i, ctx.N // 2, LO, HI) for i in range(args.batch)]
    packed = ctx.pack([ctx.encrypt(v, L, 9600 + i) for i, v in enumerate(vals)])
    for _ in range(3):
        ctx.mul(packed, packed)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, args.steps)
    e0.record(stream)
    for _ in range(reps):
        ctx.mul(packed, packed)
    e1.record(stream)
    torch.cuda.synchronize()
    hedap.profile_enable(True)
    ctx.mul(packed, packed)
    torch.cuda.synchronize()
    prof = hedap.profile_read()
    hedap.profile_enable(False)
    n_ntt, ms_ntt, by_ntt = prof["ntt"]
    if args.profile_region:
        torch.cuda.profiler.start()
        ctx.mul(packed, packed)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    print(json.dumps({"hmult": {"batch": args.batch, "level": L, "ms": e0.elapsed_time(e1) / reps,
                                "ntt_launch_groups": n_ntt, "ntt_ms": ms_ntt, "ntt_algorithmic_bytes": by_ntt,
                                "ntt_limbs": by_ntt / (16.0 * ctx.N), "ntt_shapes": ctx.ntt_get_roles()}}),
          flush=True)


def bts_profile(args):
    """One batched bootstrap (bts16 chain, full slots, batch --batch) after a warm-up, its time by kernel class
    from the library's event profiler, and the same bootstrap once more between cudaProfilerStart/Stop (for
    ncu --profile-from-start off)."""
    import torch
    from paper_2606_10477_gb300 import hedap, inputs
    p, b = inputs.PRESETS["bts16"], inputs.BTS
    stream = torch.cuda.current_stream()
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 11,
                        stream=stream.cuda_stream)
    ctx.bts_setup(b["K"], b["r"], b["deg"], b["cts"], b["stc"])
    vals = [inputs.uniform_values(5000 + i, ctx.N // 2, -0.5, 0.5) for i in range(args.batch)]
    ct = ctx.pack([ctx.encrypt(v, 1, 5100 + i) for i, v in enumerate(vals)])
    ctx.bootstrap_scaled(ct, 1)  # warm-up: keys and diagonals are built here
    torch.cuda.synchronize()
    hedap.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.bootstrap_scaled(ct, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = hedap.profile_read()
    hedap.profile_enable(False)
    torch.cuda.profiler.start()
    ctx.bootstrap_scaled(ct, 1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"bootstrap": {"batch": args.batch, "ms": e0.elapsed_time(e1),
                                    "classes": {k: {"groups": v[0], "ms": v[1]} for k, v in prof.items() if v[0]}}}),
          flush=True)


def run_ntt_only(args):
    import torch
    from paper_2606_10477_gb300 import hedap, inputs
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    p = inputs.PRESETS[PRESET]
    ctx = hedap.Context(p["log_n"], p["q_bits"], p["p_bits"], p["alpha"], p["log_scale"], p["hw"], 1,
                        stream=stream.cuda_stream)
    fwd, inv, fv, iv = ctx.ntt_tune(args.ntt_limbs, 3)
    loop = ctx.butterfly_rate() / 1e9  # the register-only butterfly loop (k_butterfly_loop), before the region
    r = measure_ntt(ctx, inputs, torch, stream, args.ntt_limbs, reps=max(1, args.steps),
                    profile_region=args.profile_region)
    print(json.dumps({"metric": "NTT GB/s (N=2^16, 64-bit limbs, batched)", "value": r["forward"]["gbs"],
                      "unit": "GB/s", "ntt": r, "tune": {"forward_ms": fwd, "inverse_ms": inv,
                                                         "chosen": [fv, iv], "roles": ctx.ntt_get_roles()},
                      "register_loop_gbutterfly_s": loop}), flush=True)


def main():
    args = parse()
    if args.only == "ntt":
        run_ntt_only(args)
    elif args.only == "hmult":
        run_hmult_only(args)
    elif args.only == "ops":
        run_ops_only(args)
    elif args.only == "serving":
        run_serving_only(args)
    elif args.only == "bts" and args.profile_region:
        bts_profile(args)
    elif args.only == "bts":
        import torch
        from paper_2606_10477_gb300 import hedap, inputs
        print(json.dumps({"bootstrapped": bootstrapped_workload(hedap.Context, inputs, torch,
                                                                torch.cuda.current_stream(), 0, args.batch)}))
    elif args.only == "mixed":
        import torch
        from paper_2606_10477_gb300 import hedap, inputs
        print(json.dumps({"mixed_levels": mixed_workload(hedap, inputs, torch, torch.cuda.current_stream(), 0)}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
