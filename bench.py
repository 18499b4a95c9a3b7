#!/usr/bin/env python3
"""Benchmark: SCOUP sparse code uplift throughput on GB300.

Workload: 1M Gaussians in 64 blobs, 200 sphere-band views at 988x731, 200
Voronoi regions per view, C=256 atoms, s=8 nonzeros per region code, K=8
(synthetic, seeded).  One step = one full uplift (all 200 views: projection,
binning, per-tile sort + composite + sparse scatter) followed by the Top-K +
L1 normalisation of every Gaussian, through the C ABI.

Metric: accepted Gaussian-pixel contributions per second (alpha >= 1/255,
before the transmittance stop), the count the library reports.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs its own replica of the workload on its GPU
(independent problems, weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "uplift Gaussian-pixel contributions/s"
UNIT = "contributions/s"
WORKLOAD = "uplift_1M_gaussians_200views_988x731_C256_s8_K8"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--views", type=int, default=200, help="views of the workload (default: all 200)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-form-compare", action="store_true",
                    help="skip timing the other uplift form beside the headline")
    ap.add_argument("--per-view", action="store_true",
                    help="time the per-view form (one tile launch per view) instead of the chunked form")
    ap.add_argument("--no-entropy", action="store_true",
                    help="skip the Top-K + entropy and entropy-filter measurement")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU oracle sample budget")
    ap.add_argument("--render-views", type=int, default=8,
                    help="views of the 1920x1080 render + decode measurement (0 = skip)")
    ap.add_argument("--dense-views", type=int, default=20,
                    help="views of the dense (D=512) vs sparse uplift comparison (0 = skip)")
    ap.add_argument("--level-views", type=int, default=20,
                    help="views of the three-level one-pass vs separate-pass comparison (0 = skip)")
    ap.add_argument("--backward-views", type=int, default=8,
                    help="views of the differentiable-render measurement (0 = skip)")
    ap.add_argument("--batch-scenes", type=int, default=16,
                    help="scenes of the batched-uplift measurement (0 = skip)")
    ap.add_argument("--decode-rows", type=int, default=0,
                    help="only time the bf16 decode GEMM on this many rows of codes (C=256, D=512) and exit")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# distributed plumbing (host-side barrier and max-over-ranks only)
# ----------------------------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, uuid: str | None):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if uuid and uuid not in parts[1]:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower().startswith("active")})
        busy = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def profiled_traffic(kernel: str, source: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or None
    when the summary is missing or was taken on a different source file."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_2605_13600_gb300", "csrc", source)
    if not os.path.exists(src):
        return None
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for path in glob.glob(os.path.join(ROOT, "profiles", f"{kernel}*.txt")):
        fields = {}
        for line in open(path):
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256") == sha and "traffic_bytes_per_launch" in fields:
            return float(fields["traffic_bytes_per_launch"])
    return None


# ----------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(budget_s: float, max_views: int = 16, device: str = "cpu"):
    """Time the FP64 oracle on the first views of the same workload, one view
    at a time, until the budget is spent.  Returns (contributions/s, views, threads)."""
    import oracle
    import synth
    oracle.build()
    threads = os.cpu_count() or 1
    wl = synth.uplift_cfg2(device=device, V=max_views)
    done_views, contrib, elapsed = 0, 0, 0.0
    for v in range(max_views):
        t0 = time.perf_counter()
        _, _, cnt = oracle.uplift(wl, views=[v], nthreads=threads)
        elapsed += time.perf_counter() - t0
        contrib += cnt["contributions"]
        done_views += 1
        if elapsed >= budget_s:
            break
    # one view on one thread: the oracle's single-core rate
    t0 = time.perf_counter()
    _, _, cnt = oracle.uplift(wl, views=[0], nthreads=1)
    single = cnt["contributions"] / (time.perf_counter() - t0)
    return contrib / elapsed, done_views, threads, elapsed, single


def cpu_model() -> str:
    """The host CPU's model name (lscpu), or the platform's processor string."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def run_reference(args, dist):
    """The oracle, as it stands, on the host cores: each step one view of the
    workload (a bounded sample); rank 0 only."""
    if dist.rank != 0:
        return
    import oracle
    import synth
    oracle.build()
    threads = os.cpu_count() or 1
    nviews = args.warmup + args.steps
    wl = synth.uplift_cfg2(device="cpu", V=nviews)
    for v in range(args.warmup):
        oracle.uplift(wl, views=[v], nthreads=threads)
    contrib, t_total = 0, 0.0
    for v in range(args.warmup, nviews):
        t0 = time.perf_counter()
        _, _, cnt = oracle.uplift(wl, views=[v], nthreads=threads)
        t_total += time.perf_counter() - t0
        contrib += cnt["contributions"]
    value = contrib / t_total
    sample = (f"one view per step (views {args.warmup}..{nviews - 1} of 200) of the 1M-Gaussian "
              f"988x731 workload, FP64 oracle, OpenMP over tiles")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "1 view per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ----------------------------------------------------------------------------
# GB300 arm
# ----------------------------------------------------------------------------

def run_gb300(args, dist):
    import numpy as np
    import torch

    import synth
    from paper_2605_13600_gb300 import build as gbuild
    gbuild.build()
    import paper_2605_13600_gb300 as gb

    dev = torch.device("cuda", dist.local if dist.world > 1 else 0)
    torch.cuda.set_device(dev)
    wl = synth.uplift_cfg2(device=str(dev), V=args.views)
    # the chunked form (SCOUP_UPLIFT_CHUNKED): chunks of 8 views on two lanes,
    # one persistent tile launch per chunk
    up = gb.Uplift(wl, device=str(dev), chunked=not args.per_view)
    st0 = up.run(stats=True)
    if st0["status"] != 0:
        raise RuntimeError(f"uplift status {st0['status']}")
    contrib = st0["contributions"]

    for _ in range(args.warmup):
        up.run(stats=False)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    clocks = ClockSampler()
    l0 = gb.scoup_launch_count()
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(args.steps):
        up.run(stats=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop(uuid)
    launches = (gb.scoup_launch_count() - l0) // args.steps
    st_end = gb.scoup_read_stats(up.workspace)
    if st_end["status"] != 0:
        raise RuntimeError(f"uplift status {st_end['status']} after the timed loop")
    t_step = ev0.elapsed_time(ev1) / 1e3 / args.steps
    t_max = dist.max(t_step)
    value = dist.world * contrib / t_max

    # end to end through the public API with host buffers (right after the device-timed
    # steps, before the profiling and roofline passes touch the GPU)
    e2e = None
    if not args.no_e2e:
        host = {
            "means": torch.as_tensor(wl.scene.means).pin_memory(),
            "scales": torch.as_tensor(wl.scene.scales).pin_memory(),
            "quats": torch.as_tensor(wl.scene.quats).pin_memory(),
            "opacity": torch.as_tensor(wl.scene.opacity).pin_memory(),
            "region_maps": torch.as_tensor(wl.region_maps).pin_memory(),
            "code_idx": torch.as_tensor(wl.code_idx).pin_memory(),
            "code_val": torch.as_tensor(wl.code_val).pin_memory(),
        }
        out_i = torch.empty(up.topk_idx.shape, dtype=torch.int32).pin_memory()
        out_v = torch.empty(up.topk_val.shape, dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = out_i.numel() * 4 + out_v.numel() * 4

        def e2e_step(chunked=None):
            # scene and code table copied up front; the region maps (93% of the
            # input bytes) staged by the library while earlier work computes
            # (scoup_uplift_host_maps in the headline's form by default)
            for k, t in host.items():
                if k != "region_maps":
                    getattr(up, k).copy_(t, non_blocking=True)
            up.run_host_maps(host["region_maps"], stats=False, chunked=chunked)
            out_i.copy_(up.topk_idx, non_blocking=True)
            out_v.copy_(up.topk_val, non_blocking=True)

        def timed_e2e(step):
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            dist.barrier()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                step()
            torch.cuda.synchronize()
            return dist.max((time.perf_counter() - t0) / args.steps)

        t_e2e = timed_e2e(e2e_step)
        t_o = timed_e2e(lambda: e2e_step(chunked=args.per_view))
        e2e = {"value": dist.world * contrib / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": t_e2e * 1e3,
               "form": "pinned host inputs; scene and codes copied, region maps staged by "
                       "scoup_uplift_host_maps in the headline's form while earlier work computes; Top-K read back",
               "other_form": {"value": dist.world * contrib / t_o, "ms_per_step": t_o * 1e3,
                              "form": "the same in the " + ("chunked" if args.per_view else "per-view") + " form"}}


    # per-phase kernel times (CUDA events on the launching stream)
    gb.scoup_profile_enable(True)
    for _ in range(2):
        up.run(stats=False)
    torch.cuda.synchronize()
    prof = gb.scoup_profile_read()
    gb.scoup_profile_enable(False)
    step_ms = {k: v[0] / 2 for k, v in prof.items()}
    tiles_ms, tiles_n = prof.get("uplift_tiles", (0.0, 1))
    per_launch_s = tiles_ms / tiles_n / 1e3

    # roofline of the dominant kernel (per-tile composite + scatter: one drain
    # launch per chunk of views, or one launch per view in the per-view form)
    pk = peaks()
    V = len(up.cams)
    views_per_launch = V / (tiles_n / 2)
    evaluated_per_launch = st0["evaluated_pairs"] / V * views_per_launch
    # FP32-pipe work of Eq. 2 for every evaluated Gaussian-pixel pair, accepted
    # or not (a lower bound for any implementation; the exp runs on the SFU and
    # is not counted, nor e = alpha T of the accepted pairs): exponent 2
    # subtractions + 3 products + 2 fused sums, 2 threshold compares, exp
    # argument scale, alpha = o exp, min with 0.99, 1 - alpha, T (1 - alpha),
    # stop compare -> 15 operations
    ops = 15.0 * evaluated_per_launch
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sms * 128 * pk["sm_max_mhz"] * 1e6  # FP32 lanes x max SM clock
    achieved = ops / per_launch_s
    npx = up.cams[0].width * up.cams[0].height
    # algorithmic HBM bytes of one view: region map + one FP32 read-modify-write per
    # accumulator update issued + one 32-byte record per visible Gaussian
    bytes_launch = (4.0 * npx + 8.0 * st0["atomics"] / V + 32.0 * st0["visible"] / V) * views_per_launch
    kname = "uplift_tile_kernel" if args.per_view else "uplift_drain_kernel"
    traffic = profiled_traffic(kname, "uplift_tile.cu")
    roofline = {"kernel": kname, "views_per_launch": views_per_launch, "bound": "alu", "achieved": achieved / 1e12,
                "peak": alu_peak / 1e12, "unit": "Tops/s (FP32 lane ops)",
                "frac": achieved / alu_peak, "traffic": traffic,
                "per_launch_ms": per_launch_s * 1e3,
                "hbm_view": {"algorithmic_bytes_per_launch": bytes_launch,
                             "achieved_gbs": bytes_launch / per_launch_s / 1e9,
                             "peak_gbs": pk["hbm_gbs"],
                             "frac": bytes_launch / per_launch_s / 1e9 / pk["hbm_gbs"]},
                "ops_per_launch": ops, "op_count": "15 FP32 ops per evaluated pair (exp on the SFU not counted)",
                "peak_source": pk["source"] + f" (HBM); FP32 lanes x max SM clock x {n_sms} SMs (ALU)"}
    roofline["step"] = step_roofline(gb, up, wl, st0, t_step, pk, alu_peak)

    # the other form on the same workload, for comparison (not the headline)
    other = None
    if not args.no_form_compare:
        upo = gb.Uplift(wl, device=str(dev), dup_capacity=up.dup_capacity, chunked=args.per_view)
        so = upo.run(stats=True)
        if so["status"] != 0 or so["contributions"] != contrib:
            raise RuntimeError("the two uplift forms disagree on the contributions")
        for _ in range(args.warmup):
            upo.run(stats=False)
        torch.cuda.synchronize()
        dist.barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            upo.run(stats=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_o = dist.max(ev0.elapsed_time(ev1) / 1e3 / args.steps)
        other = {"value": dist.world * contrib / t_o, "ms_per_step": t_o * 1e3,
                 "form": ("chunked: 8 views per chunk on two lanes, one persistent tile launch per chunk"
                          if args.per_view else "per-view: one tile launch per view, two view pipelines")}
        del upo
        torch.cuda.empty_cache()

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        v, nv, threads, el, single = oracle_sample(args.cpu_seconds, device=str(dev))
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"views 0..{nv - 1} of 200 of the same workload (all 1M Gaussians, 988x731), "
                         f"FP64 oracle, {el:.1f} s",
               "cpu_model": cpu_model(),
               "single_thread": {"value": single, "unit": UNIT, "sample": "view 0 on one thread"}}

    ent = entropy_leg(args, up, pk) if not args.no_entropy else None

    rd = None
    if args.render_views > 0:
        rd = render_decode_leg(args, dist, wl, up, dev, pk)

    dn = None
    if args.dense_views > 0:
        dn = dense_leg(args, dist, wl, up, dev)

    bw = None
    if args.backward_views > 0:
        bw = backward_leg(args, dist, dev)

    lv = None
    if args.level_views > 0:
        lv = levels_leg(args, dist, dev)

    bt = None
    if args.batch_scenes > 0:
        del up
        torch.cuda.empty_cache()
        bt = batched_leg(args, dist, dev)

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded stand-in for pretrained 3DGS scenes with SAM/CLIP region codes)",
            "config": {"workload": WORKLOAD, "n_gaussians": wl.scene.n, "views": V,
                       "width": 988, "height": 731, "regions_per_view": 200, "C": wl.C, "s": wl.s,
                       "K": wl.K, "contributions_per_step": contrib,
                       "evaluated_pairs_per_step": st0["evaluated_pairs"],
                       "l2": "inputs larger than L2 (region maps 578 MB, accumulator 1.02 GB)",
                       "parallelism": f"replica x{dist.world}"},
            "form": ("per-view: one tile launch per view, two view pipelines" if args.per_view else
                     "chunked (SCOUP_UPLIFT_CHUNKED): 8 views per chunk on two lanes, one persistent tile "
                     "launch per chunk"),
            "other_form": other,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "phase_ms_per_step": step_ms,
            "stats": {k: st0[k] for k in ("visible", "duplicates", "flushes", "atomics")},
            "entropy": ent,
            "render_decode": rd,
            "dense_vs_sparse": dn,
            "levels": lv,
            "render_backward": bw,
            "batched": bt,
        }
        print(json.dumps(line), flush=True)


def render_decode_leg(args, dist, wl, up, dev, pk):
    """Secondary measurement: sparse-code rendering (Eq. 7) of 1920x1080 views of
    the same 1M Gaussians with the Top-K codes the uplift just produced, codebook
    decode (Eq. 8) to bf16 features and cosine similarity to 32 text vectors,
    the similarity computed in the decode GEMM (scoup_decode_query).  Returns
    the MPix/s figure with its phase split, the decode GEMM roofline and the
    three-call form (render, scoup_decode, scoup_similarity) beside it."""
    import numpy as np
    import torch

    import synth
    import paper_2605_13600_gb300 as gb

    rw = synth.render_cfg4(n_views=args.render_views)
    cams = rw.cams
    ren = gb.Render(wl.scene, up.topk_idx.cpu().numpy(), up.topk_val.cpu().numpy(), wl.C, cams,
                    device=str(dev))
    H, W = cams[0].height, cams[0].width
    P = H * W
    D, Q = rw.codebook.shape[1], rw.text.shape[0]
    out = ren.outputs(cams[0], dtype=torch.bfloat16)  # bf16 codes: the decode's input type
    codebook = torch.from_numpy(rw.codebook).to(dev)
    text = torch.from_numpy(rw.text).to(dev)
    feats = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    n2 = torch.empty((P,), dtype=torch.float32, device=dev)
    sim = torch.empty((P, Q), dtype=torch.float32, device=dev)
    dws = torch.empty(gb.scoup_decode_workspace_size(P, wl.C, D), dtype=torch.uint8, device=dev)
    sws = torch.empty(gb.scoup_similarity_workspace_size(P, D, Q), dtype=torch.uint8, device=dev)
    qws = torch.empty(gb.scoup_decode_query_workspace_size(P, wl.C, D, Q), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def view(v):
        ren.run(v, out=out, stats=False)
        gb.scoup_decode_query(out[0].view(P, wl.C), codebook, text, sim, features=feats, feat_norm2=n2,
                              workspace=qws)

    def view_three(v):
        ren.run(v, out=out, stats=False)
        gb.scoup_decode(out[0].view(P, wl.C), codebook, feats, n2, workspace=dws)
        gb.scoup_similarity(feats, text, sim, feat_norm2=n2, workspace=sws)

    stats = [ren.run(v, out=out, stats=True)[1] for v in range(len(cams))]
    for st in stats:
        if st["status"] != 0:
            raise RuntimeError(f"render status {st['status']}")
    for _ in range(max(3, args.warmup)):
        view(0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for v in range(len(cams)):
        view(v)
    ev1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    t = dist.max(ev0.elapsed_time(ev1) / 1e3)
    mpix = dist.world * len(cams) * P / t / 1e6

    gb.scoup_profile_enable(True)
    for v in range(len(cams)):
        view(v)
    torch.cuda.synchronize()
    prof = gb.scoup_profile_read()
    gb.scoup_profile_enable(False)
    phase_ms = {k: prof[k][0] / len(cams) for k in ("render", "decode", "similarity") if k in prof}
    if "decode" in phase_ms:
        phase_ms["decode_with_similarity"] = phase_ms.pop("decode")
    if gb.scoup_read_stats(qws)["status"] != 0:
        raise RuntimeError("decode + query device status")

    # the three-call form: render, decode, similarity (the features read back)
    for _ in range(3):
        view_three(0)
    torch.cuda.synchronize()
    ev0.record(stream)
    for v in range(len(cams)):
        view_three(v)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_three = ev0.elapsed_time(ev1) / 1e3
    gb.scoup_profile_enable(True)
    for v in range(len(cams)):
        view_three(v)
    torch.cuda.synchronize()
    prof3 = gb.scoup_profile_read()
    gb.scoup_profile_enable(False)
    phase3 = {k: prof3[k][0] / len(cams) for k in ("render", "decode", "similarity") if k in prof3}
    if gb.scoup_read_stats(dws)["status"] != 0 or gb.scoup_read_stats(sws)["status"] != 0:
        raise RuntimeError("decode/similarity device status")

    # the same views through the one-call form (scoup_render_decode_fused) + similarity
    def view_fused(v):
        ren.run_decode(v, codebook, feats, n2, stats=False)
        gb.scoup_similarity(feats, text, sim, feat_norm2=n2, workspace=sws)

    for _ in range(3):
        view_fused(0)
    torch.cuda.synchronize()
    ev0.record(stream)
    for v in range(len(cams)):
        view_fused(v)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_fused = ev0.elapsed_time(ev1) / 1e3
    if ren.run_decode(0, codebook, feats, n2, stats=True)["status"] != 0:
        raise RuntimeError("fused render+decode status")

    # relevancy (App. B, Eq. 9) of 28 queries against 4 canonical phrases from the last view's similarities
    Rel = torch.empty((P, Q - 4), dtype=torch.float32, device=dev)
    for _ in range(3):
        gb.scoup_relevancy(sim, 4, Rel)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(10):
        gb.scoup_relevancy(sim, 4, Rel)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_rel = ev0.elapsed_time(ev1) / 1e3 / 10
    rel_bytes = 4.0 * P * Q + 4.0 * P * (Q - 4)
    # similarity + relevancy as two calls vs relevancy in the similarity GEMM's epilogue
    rws = gb.scoup_similarity_relevancy(feats, text, 4, Rel, feat_norm2=n2)

    def time_reps(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps

    t_two = time_reps(lambda: (gb.scoup_similarity(feats, text, sim, feat_norm2=n2, workspace=sws),
                               gb.scoup_relevancy(sim, 4, Rel)))
    t_epi = time_reps(lambda: gb.scoup_similarity_relevancy(feats, text, 4, Rel, feat_norm2=n2, workspace=rws))
    epi_bytes = 2.0 * P * D + 4.0 * P * (Q - 4)  # bf16 features in, relevancy out
    # decode + similarity + relevancy: three calls vs one decode GEMM whose query unit writes the relevancy
    codes_v = out[0].view(P, wl.C)
    t_dsr = time_reps(lambda: (gb.scoup_decode(codes_v, codebook, feats, n2, workspace=dws),
                               gb.scoup_similarity(feats, text, sim, feat_norm2=n2, workspace=sws),
                               gb.scoup_relevancy(sim, 4, Rel)))
    t_qrel = time_reps(lambda: gb.scoup_decode_query(codes_v, codebook, text, Rel, n_canon=4, features=feats,
                                                     feat_norm2=n2, workspace=qws))
    t_qrel_nf = time_reps(lambda: gb.scoup_decode_query(codes_v, codebook, text, Rel, n_canon=4,
                                                        workspace=qws))

    # the decode GEMM alone: bf16 codes in, bf16 features out (one launch + a 256x512 transpose)
    codes_bf16 = out[0].view(P, wl.C)
    for _ in range(3):
        gb.scoup_decode(codes_bf16, codebook, feats, n2, workspace=dws)
    torch.cuda.synchronize()
    reps = 10
    ev0.record(stream)
    for _ in range(reps):
        gb.scoup_decode(codes_bf16, codebook, feats, n2, workspace=dws)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_gemm = ev0.elapsed_time(ev1) / 1e3 / reps
    flops = 2.0 * P * wl.C * D
    gemm_bytes = 2.0 * P * wl.C + 2.0 * P * D
    # the same GEMM with the query unit: + 4 Q bytes of similarities written per pixel
    t_query = time_reps(lambda: gb.scoup_decode_query(codes_bf16, codebook, text, sim, features=feats,
                                                      feat_norm2=n2, workspace=qws))
    query_bytes = gemm_bytes + 4.0 * P * Q
    evaluated = sum(s["evaluated_pairs"] for s in stats) / len(stats)
    contrib = sum(s["contributions"] for s in stats) / len(stats)
    return {
        "metric": "render+decode+similarity pixels/s", "value": mpix, "unit": "MPix/s",
        "workload": rw.name, "views_timed": len(cams), "pixels_per_view": P,
        "C": wl.C, "D": D, "Q": Q, "K": wl.K,
        "codes": "Top-K of the uplift measured above",
        "ms_per_view": t * 1e3 / len(cams), "phase_ms_per_view": phase_ms,
        "relevancy": {"ms_per_view": t_rel * 1e3, "queries": Q - 4, "canonical": 4, "bound": "hbm",
                      "achieved": rel_bytes / t_rel / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                      "frac": rel_bytes / t_rel / 1e9 / pk["hbm_gbs"],
                      "similarity_then_relevancy_ms": t_two * 1e3,
                      "epilogue_form": {"call": "scoup_similarity_relevancy", "ms_per_view": t_epi * 1e3,
                                        "bound": "hbm", "achieved": epi_bytes / t_epi / 1e9,
                                        "peak": pk["hbm_gbs"], "unit": "GB/s",
                                        "frac": epi_bytes / t_epi / 1e9 / pk["hbm_gbs"],
                                        "speedup_vs_two_calls": t_two / t_epi},
                      "decode_epilogue_form": {"call": "scoup_decode_query (n_canon 4)",
                                               "decode_similarity_relevancy_ms": t_dsr * 1e3,
                                               "ms_per_view": t_qrel * 1e3,
                                               "speedup_vs_three_calls": t_dsr / t_qrel,
                                               "without_features_ms": t_qrel_nf * 1e3}},
        "form": "render -> scoup_decode_query (bf16 features, norms and the similarities from one GEMM)",
        "three_call_form": {"form": "render -> scoup_decode -> scoup_similarity",
                            "value": len(cams) * P / t_three / 1e6, "unit": "MPix/s",
                            "ms_per_view": t_three * 1e3 / len(cams), "phase_ms_per_view": phase3},
        "fused_call": {"form": "scoup_render_decode_fused + scoup_similarity",
                       "value": len(cams) * P / t_fused / 1e6, "unit": "MPix/s",
                       "ms_per_view": t_fused * 1e3 / len(cams)},
        "render_evaluated_pairs_per_view": evaluated, "render_contributions_per_view": contrib,
        # the decode GEMM moves more bytes than its FLOPs need time for at these
        # shapes (t_hbm = 2(C + D) B/pixel / BW > t_tensor = 2 C D / peak), so its
        # roofline is HBM: algorithmic bytes = bf16 codes read + bf16 features written
        "decode_roofline": {"kernel": "gemm_bf16_kernel", "bound": "hbm",
                            "achieved": gemm_bytes / t_gemm / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                            "frac": gemm_bytes / t_gemm / 1e9 / pk["hbm_gbs"],
                            "algorithmic_bytes_per_launch": gemm_bytes, "per_launch_ms": t_gemm * 1e3,
                            "tensor_view": {"achieved_tflops": flops / t_gemm / 1e12, "peak_tflops": pk["bf16_tflops"],
                                            "frac": flops / t_gemm / 1e12 / pk["bf16_tflops"]},
                            "peak_source": pk["source"] + " (HBM copy; bf16 burst)"},
        "decode_query_roofline": {"kernel": "gemm_bf16_kernel (with the query unit)", "bound": "hbm",
                                  "achieved": query_bytes / t_query / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                  "frac": query_bytes / t_query / 1e9 / pk["hbm_gbs"],
                                  "algorithmic_bytes_per_launch": query_bytes, "per_launch_ms": t_query * 1e3,
                                  "vs_decode_then_similarity_ms": (t_gemm * 1e3,
                                                                   phase3.get("similarity", float("nan")))},
    }


def red_ceiling(gb, log2_n: int = 29, count: int = 1 << 28, reps: int = 3):
    """Measured FP32 atomic-update throughput (updates/s): `count` reductions
    to pseudo-random elements of a 2^log2_n-float buffer (2 GB, far larger
    than L2), best of `reps` runs timed with CUDA events."""
    import torch
    buf = torch.zeros(1 << log2_n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    gb.scoup_selftest_red_throughput(buf, count // 4, seed=7)  # warm-up
    best = None
    for r in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gb.scoup_selftest_red_throughput(buf, count, seed=11 + r)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    del buf
    torch.cuda.empty_cache()
    return count / best


def step_roofline(gb, up, wl, st0, t_step, pk, alu_peak):
    """The uplift step against its three ceilings (HBM bytes, atomic updates,
    FP32 ALU), with the method's algorithmic work:
      bytes   = sum_v (44 N + 4 H W + 8 U_v) + 4 N C + 8 N K
                (parameters read per view, region map, one read-modify-write
                per distinct (Gaussian, atom) updated in view v, the final
                accumulator read and the Top-K write);
      atomics = sum_v U_v (lower bound; the issued count and s x contributions
                of Algorithm 1 are reported beside it);
      ALU     = 15 FP32 operations per evaluated (Gaussian, pixel) pair.
    U_v is counted exactly: view v alone is uplifted into a cleared
    accumulator and its non-zero entries are counted."""
    import torch
    n, C, K, s = wl.scene.n, wl.C, wl.K, wl.s
    V = len(up.cams)
    U = []
    for v in range(V):
        up.run(stats=False, views=[v], topk=False)
        U.append(int(torch.count_nonzero(up.accum).item()))
    up.run(stats=False)  # the later legs start from the full step's accumulator
    pix = sum(c.width * c.height for c in up.cams)
    sum_u = float(sum(U))
    bytes_step = 44.0 * n * V + 4.0 * pix + 8.0 * sum_u + 4.0 * n * C + 8.0 * n * K
    red = red_ceiling(gb)
    t_hbm = bytes_step / (pk["hbm_gbs"] * 1e9)
    t_atom = sum_u / red
    t_alu = 15.0 * st0["evaluated_pairs"] / alu_peak
    t_roof = max(t_hbm, t_atom)
    ceilings = {"hbm": t_hbm, "atomic": t_atom, "alu": t_alu}
    return {"ms_per_step": t_step * 1e3,
            "bytes_per_step": bytes_step, "hbm_ms": t_hbm * 1e3, "hbm_frac": t_hbm / t_step,
            "atomics_lower_bound": sum_u, "atomics_issued": float(st0["atomics"]),
            "atomics_alg1_literal": float(s) * st0["contributions"],
            "red_peak_per_s": red, "red_peak_source": "measured: scoup_selftest_red_throughput, 2^28 FP32 "
                                                      "reductions over a 2 GB buffer, best of 3",
            "atomic_ms": t_atom * 1e3, "atomic_frac": t_atom / t_step,
            "alu_ms": t_alu * 1e3, "alu_frac": t_alu / t_step,
            "roofline_ms": t_roof * 1e3, "frac": t_roof / t_step,
            "binding": max(ceilings, key=ceilings.get),
            "formula": "t_roof = max(bytes / HBM, sum_v U_v / RED peak); ALU (15 ops per evaluated pair) beside it"}


def entropy_leg(args, up, pk):
    """Top-K with the coefficient entropy fused in, and the entropy filter,
    at full size on the accumulator the uplift just produced (1M x 256)."""
    import torch

    import paper_2605_13600_gb300 as gb
    n, C = up.accum.shape[-2], up.accum.shape[-1]
    K = up.K
    acc = up.accum if up.accum.dim() == 2 else up.accum[0]
    dev = acc.device
    idx = torch.empty((n, K), dtype=torch.int32, device=dev)
    val = torch.empty((n, K), dtype=torch.float32, device=dev)
    H = torch.empty((n,), dtype=torch.float32, device=dev)
    mask = torch.empty((n,), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / 1e3 / reps

    t_topk = timed(lambda: gb.scoup_topk(acc, K, idx, val))
    t_ent = timed(lambda: gb.scoup_topk_entropy(acc, K, idx, val, H))
    # the filter runs on the stream without host round-trips: timed like the rest
    from paper_2605_13600_gb300._lib import load
    ws = torch.empty(int(load().scoup_entropy_filter_workspace_size()), dtype=torch.uint8, device=dev)
    t_filter = timed(lambda: gb.scoup_entropy_filter(H, n // 2, idx, val, mask, workspace=ws), reps=5)
    kept = int(mask.sum().item())
    nbytes = 4.0 * n * C + 8.0 * n * K
    return {
        "rows": n, "C": C, "K": K,
        "topk_ms": t_topk * 1e3,
        "topk_entropy_ms": t_ent * 1e3,
        "topk_entropy_roofline": {"bound": "hbm", "achieved": (nbytes + 4.0 * n) / t_ent / 1e9,
                                  "peak": pk["hbm_gbs"], "unit": "GB/s",
                                  "frac": (nbytes + 4.0 * n) / t_ent / 1e9 / pk["hbm_gbs"],
                                  "algorithmic_bytes": nbytes + 4.0 * n},
        "entropy_filter_ms": t_filter * 1e3, "entropy_filter_keep": n // 2, "entropy_filter_kept": kept,
        "entropy_filter_form": "8 radix-select passes over the entropies, each digit picked on the device (no host round-trip)",
    }


def dense_leg(args, dist, wl, up, dev):
    """Secondary measurement: the dense feature uplift of Eq. 3 (a 512-d unit
    feature per region, plus the normaliser Z) against the sparse uplift
    (s = 8 entries per region) on the same views, both accumulate-only: the
    time ratio the paper's O(|S_i| D) -> O(|S_i| K) argument predicts."""
    import torch

    import synth
    import paper_2605_13600_gb300 as gb

    views = range(min(args.dense_views, len(up.cams)))
    dwl = synth.dense_feature_codes(wl, D=512, seed=7)
    dup = gb.Uplift(dwl, device=str(dev), topk=False)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for name, u in (("sparse_s8", up), ("dense_d512", dup)):
        st = u.run(stats=True, views=views, topk=False)
        if st["status"] != 0:
            raise RuntimeError(f"{name} status {st['status']}")
        u.run(stats=False, views=views, topk=False)
        torch.cuda.synchronize()
        dist.barrier()
        ev0.record(stream)
        for _ in range(2):
            u.run(stats=False, views=views, topk=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        t = dist.max(ev0.elapsed_time(ev1) / 1e3 / 2)
        out[name] = {"ms": t * 1e3, "contributions_per_s": dist.world * st["contributions"] / t,
                     "accumulator_atomics": st["atomics"], "entries_per_region": u.s}
    del dup
    torch.cuda.empty_cache()
    return {"views": len(views), "workload": WORKLOAD, "accumulate_only": True, **out,
            "time_ratio_dense_over_sparse": out["dense_d512"]["ms"] / out["sparse_s8"]["ms"]}


def backward_leg(args, dist, dev):
    """Secondary measurement: the differentiable sparse render workload
    (500k Gaussians, 32 views at 800x600, K = 8 of C = 256,
    a 256 x 512 codebook) with its own uplift: the scene's region codes are
    uplifted over its 32 views (scoup_uplift, outside the timed region), and
    per view the whole loss chain runs in the library -- render (Eq. 7) ->
    bf16 decode (Eq. 8) -> L2 loss against the decoded region codes and its
    gradient -> dL/dWhat = dL/dF C^T on the tensor cores -> render backward to
    the Top-K values and opacities.  MPix/s of the chain."""
    import torch

    import synth
    import paper_2605_13600_gb300 as gb

    wl, codebook = synth.uplift_cfg5(device=str(dev))
    up = gb.Uplift(wl, device=str(dev))
    st = up.run(stats=True)
    if st["status"] != 0:
        raise RuntimeError(f"cfg5 uplift status {st['status']}")
    cams = wl.cams[:max(1, args.backward_views)]
    topk_idx, topk_val = up.topk_idx.cpu().numpy(), up.topk_val.cpu().numpy()
    del up
    torch.cuda.empty_cache()
    ren = gb.Render(wl.scene, topk_idx, topk_val, wl.C, cams, device=str(dev))
    H, W = cams[0].height, cams[0].width
    P, C = H * W, wl.C
    cb = torch.as_tensor(codebook, device=dev)
    D = cb.shape[1]
    maps = torch.as_tensor(wl.region_maps, device=dev)
    ci = torch.as_tensor(wl.code_idx, device=dev)
    cv = torch.as_tensor(wl.code_val, device=dev)
    out = ren.outputs(cams[0])
    feats = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    dF = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    dW = torch.empty((H, W, C), dtype=torch.float32, device=dev)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    d_val = torch.zeros_like(ren.topk_val)
    d_op = torch.zeros_like(ren.opacity)
    dws = gb.scoup_decode(out[0].view(P, C), cb, feats)
    lws = gb.scoup_region_l2_grad(feats, maps[:P], ci, cv, cb, dF, loss)
    bws = gb.scoup_decode_backward(dF, cb, dW.view(P, C))
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def view(v):
        cam = cams[v]
        o = int(wl.map_offsets[v])
        gb.scoup_render(ren.scene, ren.topk_idx, ren.topk_val, ren.K, ren.C, cam, out[0], out[1], out[2],
                        ren.workspace, stats=False)
        gb.scoup_decode(out[0].view(P, C), cb, feats, workspace=dws)
        gb.scoup_region_l2_grad(feats, maps[o:o + P], ci, cv, cb, dF, loss, workspace=lws)
        gb.scoup_decode_backward(dF, cb, dW.view(P, C), workspace=bws)
        gb.scoup_render_backward(ren.scene, ren.topk_idx, ren.topk_val, ren.K, ren.C, cam, dW, d_val, d_op,
                                 ren.workspace)

    for _ in range(max(2, args.warmup)):
        view(0)
    torch.cuda.synchronize()
    dist.barrier()
    loss.zero_()
    ev[0].record(stream)
    for v in range(len(cams)):
        view(v)
    ev[1].record(stream)
    torch.cuda.synchronize()
    t = dist.max(ev[0].elapsed_time(ev[1]) / 1e3)
    loss_val = float(loss.item())
    gb.scoup_profile_enable(True)
    for v in range(len(cams)):
        view(v)
    torch.cuda.synchronize()
    prof = gb.scoup_profile_read()
    gb.scoup_profile_enable(False)
    for w in (ren.workspace, dws, lws, bws):
        if gb.scoup_read_stats(w)["status"] != 0:
            raise RuntimeError("loss chain device status")
    return {"metric": "render+decode+loss+backward pixels/s", "value": dist.world * len(cams) * P / t / 1e6,
            "unit": "MPix/s", "workload": wl.name, "views_timed": len(cams), "pixels_per_view": P,
            "C": C, "D": D, "K": wl.K, "ms_per_view": t * 1e3 / len(cams),
            "phase_ms_per_view": {k: prof[k][0] / len(cams) for k in ("render", "decode", "render_bwd") if k in prof},
            "loss_per_view": loss_val / len(cams),
            "chain": "scoup_render -> scoup_decode (bf16) -> scoup_region_l2_grad -> scoup_decode_backward "
                     "(bf16 tensor cores) -> scoup_render_backward",
            "codes": "Top-K of the workload's own uplift (32 views, 200 regions per view, s = 8)"}


def levels_leg(args, dist, dev):
    """Secondary measurement: three nested semantic levels (50 / 100 / 200
    regions per view, C = 256, s = 8, K = 8 each) over the 1M Gaussians, as one
    scoup_uplift_levels pass vs three scoup_uplift passes (both with Top-K)."""
    import torch

    import synth
    import paper_2605_13600_gb300 as gb

    base = synth.uplift_cfg2(device=str(dev), V=args.level_views)
    wls = synth.level_workloads(base, R_levels=(50, 100, 200), seed=11, device=str(dev))
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        dist.barrier()
        ev0.record(stream)
        for _ in range(2):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return dist.max(ev0.elapsed_time(ev1) / 1e3 / 2)

    lu = gb.LevelUplift(wls, device=str(dev))
    st = lu.run(stats=True)
    if st["status"] != 0:
        raise RuntimeError("levels status")
    t_one = timed(lambda: lu.run(stats=False))
    del lu
    ups = [gb.Uplift(wl, device=str(dev)) for wl in wls]
    t_sep = timed(lambda: [u.run(stats=False) for u in ups])
    del ups
    torch.cuda.empty_cache()
    return {"views": args.level_views, "levels": [50, 100, 200], "contributions_per_level": st["contributions"],
            "one_pass_ms": t_one * 1e3, "separate_passes_ms": t_sep * 1e3, "speedup": t_sep / t_one,
            "level_contributions_per_s_one_pass": dist.world * 3 * st["contributions"] / t_one}


def batched_leg(args, dist, dev):
    """Secondary measurement: 16 scenes of uneven size (200k-2M Gaussians,
    50-300 views, 640x480 to 1296x968), uplifted (a) as per-scene plain calls
    one after another on one stream and (b) as one autotuned batch replayed
    from a CUDA graph.  Same metric as the headline (contributions/s)."""
    import torch

    import synth
    import paper_2605_13600_gb300 as gb

    t_gen = time.perf_counter()
    wls = [synth.uplift_cfg3_scene(b, device=str(dev)) for b in range(args.batch_scenes)]
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(1, min(args.steps, 3))

    # (a) plain: one scoup_uplift per scene, back to back
    ups = [gb.Uplift(wl, device=str(dev)) for wl in wls]
    sts = [u.run(stats=True) for u in ups]
    contrib = sum(st["contributions"] for st in sts)
    for u in ups:
        u.run(stats=False)
    torch.cuda.synchronize()
    dist.barrier()
    ev0.record(stream)
    for _ in range(reps):
        for u in ups:
            u.run(stats=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_plain = dist.max(ev0.elapsed_time(ev1) / 1e3 / reps)
    del ups
    torch.cuda.empty_cache()

    # (b) batched: plan, autotune on 4 views per scene (scenes on lanes and the
    # chunked form), then the graph replay of the best configuration of each form
    bu = gb.BatchedUplift(wls, device=str(dev))
    t_tune = time.perf_counter()
    info = bu.autotune(sample_views=4)
    t_tune = time.perf_counter() - t_tune
    tuned = (info["lanes"], info["warp_w"], info["chunk_views"])

    def timed_form(lanes, warp_w, chunk):
        bu.set(lanes, warp_w)
        bu.set_chunk(chunk)
        bu.run()
        st_b = bu.stats()
        if any(s["status"] != 0 for s in st_b):
            raise RuntimeError("batched uplift status")
        contrib_b = sum(s["contributions"] for s in st_b)
        bu.run()
        torch.cuda.synchronize()
        dist.barrier()
        l0 = gb.scoup_launch_count()
        ev0.record(stream)
        for _ in range(reps):
            bu.run()
        ev1.record(stream)
        torch.cuda.synchronize()
        t = dist.max(ev0.elapsed_time(ev1) / 1e3 / reps)
        launches = (gb.scoup_launch_count() - l0) // reps
        fi = bu.info()
        return {"value": dist.world * contrib_b / t, "ms_per_batch": t * 1e3, "lanes": lanes, "warp_w": warp_w,
                "chunk_views": chunk, "graph_kernels": fi["graph_kernels"], "gpu_launches": int(launches),
                "contributions": contrib_b}

    def best_of(entries):
        e = min(entries, key=lambda t: t["ms"])
        return e["lanes"], e["warp_w"], e["chunk_views"]

    lanes_cfg = best_of([t for t in info["tune"] if t["chunk_views"] == 0])
    chunk_cfg = best_of([t for t in info["tune"] if t["chunk_views"] > 0])
    lanes_form = timed_form(*lanes_cfg)
    lanes_form["form"] = "scoup_uplift_batched, scenes on lanes: per-view launches, one CUDA graph launch"
    chunk_form = timed_form(*chunk_cfg)
    chunk_form["form"] = ("scoup_uplift_batched, chunked: views of all scenes in chunks, one persistent tile "
                          "launch per chunk, one CUDA graph launch")
    best = chunk_form if chunk_form["ms_per_batch"] < lanes_form["ms_per_batch"] else lanes_form
    bu.close()
    return {
        "metric": METRIC, "unit": UNIT,
        "workload": f"uplift_batch_{len(wls)}scenes_200k-2M_50-300views_640x480-1296x968_C256_s8_K8",
        "scenes": [w.name for w in wls], "views": sum(len(w.cams) for w in wls),
        "gaussians": sum(w.scene.n for w in wls), "contributions": contrib,
        "plain": {"value": dist.world * contrib / t_plain, "ms_per_batch": t_plain * 1e3,
                  "form": "one scoup_uplift per scene, back to back on one stream"},
        "batched": dict(best, tune=info["tune"], tune_s=t_tune, tuned=list(tuned)),
        "batched_lanes": lanes_form, "batched_chunked": chunk_form,
        "speedup": t_plain * 1e3 / best["ms_per_batch"],
        "speedup_chunked": t_plain * 1e3 / chunk_form["ms_per_batch"],
        "timed_batches": reps, "generation_s": t_gen,
    }


def decode_only(args):
    """The decode GEMM alone on `--decode-rows` rows of seeded sparse bf16 codes
    (C = 256 atoms, D = 512): a small case for kernel profiles."""
    import numpy as np
    import torch

    import synth
    import paper_2605_13600_gb300 as gb
    from paper_2605_13600_gb300 import build as gbuild
    gbuild.build()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(4)
    P, C, D = args.decode_rows, 256, 512
    codebook = torch.from_numpy(synth.unit_rows(rng, C, D)).to(dev)
    codes = torch.zeros((P, C), dtype=torch.float32, device=dev)
    idx = torch.randint(0, C, (P, 8), device=dev, generator=torch.Generator(device=dev).manual_seed(4))
    codes.scatter_(1, idx, torch.rand((P, 8), device=dev, generator=torch.Generator(device=dev).manual_seed(5)))
    codes = codes.to(torch.bfloat16)
    feats = torch.empty((P, D), dtype=torch.bfloat16, device=dev)
    n2 = torch.empty((P,), dtype=torch.float32, device=dev)
    ws = torch.empty(gb.scoup_decode_workspace_size(P, C, D), dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        gb.scoup_decode(codes, codebook, feats, n2, workspace=ws)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        gb.scoup_decode(codes, codebook, feats, n2, workspace=ws)
    ev1.record()
    torch.cuda.synchronize()
    if gb.scoup_read_stats(ws)["status"] != 0:
        raise RuntimeError("decode status")
    t = ev0.elapsed_time(ev1) / 1e3 / args.steps
    nbytes = 2.0 * P * (C + D)
    print(json.dumps({"decode_rows": P, "ms_per_launch": t * 1e3, "gbs": nbytes / t / 1e9,
                      "tflops": 2.0 * P * C * D / t / 1e12}), flush=True)


def main():
    args = parse_args()
    if args.decode_rows > 0:
        decode_only(args)
        return
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_gb300(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
