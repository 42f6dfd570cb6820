#!/usr/bin/env python
"""Benchmark: multiple-precision GEMM on one GB300 (arXiv 1410.1599 Sec. 3
workload shape), printed as one JSON line.

Step = one C := A B of the chosen algorithm (default: Winograd's variant,
n = 2048, 512-bit mantissas, cutoff 64, odd sizes peeled, entries
U[-1,1) * 2^e with e uniform in [-16, 16]).  value = effective MP GFLOP/s,
2 m l n / t, over all ranks (each rank multiplies its own matrices: replicas,
weak scaling).  Inputs (2 x 306 MB at 512 bits) exceed the 129 MB L2.

--impl reference times the CPU oracle (plain C, the tests' reference) on a
bounded sample of the same workload instead.
"""
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

ALGO_NAMES = {"simple": 0, "block": 1, "strassen": 2, "winograd": 3}
# DRAM bytes (read + write) of one leaf launch of the 512-bit Winograd product
# with cutoff 64, per 64^3 leaf: one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of the current leaf kernel (TMA-staged, slabs of 8)
# at n = 1024 (2401 leaves, 1.443 + 0.694 = 2.137 GB), scaled by the leaves of
# a launch.  Reset to None whenever the leaf kernel changes.
LEAF_TRAFFIC_PER_LEAF_P512_C64 = 2.137e9 / 2401
PEAK_IMAD_PER_CLK_PER_SM = 64      # 32-bit integer multiply-add lanes per SM per clock
# the kernels behind the library's profiler classes of the GEMM leaf
KERNEL_OF_CLASS = {"leaf_tma": "gemm_block_tma_kernel",
                   "leaf_gemm": "gemm_block_sm_kernel / gemm_block_leaf_views_kernel",
                   "simple_gemm": "gemm_simple_kernel"}
SM_COUNT_GB300 = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="winograd", choices=list(ALGO_NAMES))
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--prec", type=int, default=512)
    ap.add_argument("--cutoff", type=int, default=64)
    ap.add_argument("--leaf-tma", type=int, default=1, choices=[0, 1],
                    help="stage the Block leaves' tiles with TMA (1, the library default) or thread loads (0)")
    ap.add_argument("--no-extras", action="store_true", help="skip the other algorithms and the CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--lu-n", type=int, default=1024)
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve", action="store_true", help="only the serving run (its own JSON line)")
    ap.add_argument("--configs", action="store_true",
                    help="only the other configurations' runs and the per-algorithm errors")
    ap.add_argument("--lu", action="store_true",
                    help="only the LU runs: n = --lu-n at 256 and 1024 bits, well-conditioned and Lotkin")
    ap.add_argument("--lotkin", action="store_true",
                    help="only the Lotkin LU at 8192 and 8650 bits (n = --lu-n)")
    ap.add_argument("--lu-sweep", action="store_true",
                    help="only the paper's LU experiment: no pivoting, K = 32 alpha, alpha = 1..10")
    ap.add_argument("--paper", action="store_true",
                    help="only the paper's Section 4 benchmark (sqrt matrices, Tables 2-5 shapes)")
    ap.add_argument("--cond", action="store_true",
                    help="only cond_1 of the 1024 x 1024 Lotkin matrix from its GPU inverse at 5376 bits")
    ap.add_argument("--split", action="store_true",
                    help="only the split-form comparison (4096^3 at 1024 bits by default)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Replicas:
    """N independent replicas of the workload, one per rank (the product does
    not shard: each rank multiplies its own matrices).  Nothing crosses ranks
    on the data path; the only collectives are the timing barrier and the max
    of the per-rank step time, and the reported value is the whole job's:
    world x (work per rank) / (slowest rank's time)."""

    def __init__(self, rank, world, backend="nccl", device="cuda"):
        self.rank, self.world, self.backend, self.device = rank, world, backend, device

    def init(self, local=0):
        if self.world > 1:
            import torch
            import torch.distributed as dist
            if self.backend == "nccl":
                dist.init_process_group("nccl", device_id=torch.device("cuda", local))
            else:
                dist.init_process_group(self.backend)

    def seeds(self):
        """Input seeds of this rank's A and B: every replica has its own data."""
        return 3 + 1000 * self.rank, 4 + 1000 * self.rank

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def allmax(self, x):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def whole_job(self, work_per_rank, seconds):
        """Aggregate rate over all ranks, from the slowest rank's time."""
        return self.world * work_per_rank / seconds

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def leaf_traffic(a):
    """DRAM bytes of one leaf launch for the captured configuration, else None."""
    if LEAF_TRAFFIC_PER_LEAF_P512_C64 is None:
        return None
    if a.prec != 512 or a.cutoff != 64 or a.algo not in ("strassen", "winograd"):
        return None
    n, leaves = a.n, 1
    while n > a.cutoff and n % 2 == 0:
        n //= 2
        leaves *= 7
    if n != 64:
        return None
    return round(leaves * LEAF_TRAFFIC_PER_LEAF_P512_C64)


def workload_config(a):
    return {"workload": "mp_gemm_%s_n%d_p%d_cutoff%d" % (a.algo, a.n, a.prec, a.cutoff),
            "m": a.n, "l": a.n, "n": a.n, "prec_bits": a.prec, "algo": a.algo,
            "cutoff": a.cutoff, "odd": "peel", "entries": "U[-1,1)*2^e, e~U{-16..16}",
            "l2": "inputs larger than L2 (no flush)"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # nvidia-smi's start-up can stall the driver: wait for its first sample
        t0 = time.time()
        while time.time() - t0 < 10.0:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def run_ours(a, rank, world, local):
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import build as libbuild
    from paper_1410_1599_gb300 import inputs as gen

    libbuild.build()
    torch.cuda.set_device(local)
    rep = Replicas(rank, world)
    rep.init(local)
    barrier, allmax = rep.barrier, rep.allmax

    n, p, cutoff, algo = a.n, a.prec, a.cutoff, ALGO_NAMES[a.algo]
    flops = 2.0 * n * n * n
    seed_a, seed_b = rep.seeds()
    A = gen.uniform_pm1(n, n, p, seed_a, -16, 16)
    B = gen.uniform_pm1(n, n, p, seed_b, -16, 16)
    dA, dB = mp.DeviceMP.from_host(A), mp.DeviceMP.from_host(B)
    dC = mp.DeviceMP.empty(n, n, p)
    stream = torch.cuda.Stream()
    mp.set_stream(stream)
    mp.set_leaf_tma(bool(a.leaf_tma))
    ws_bytes = mp.workspace_size(n, n, n, p, algo, cutoff)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device="cuda")
    mp.set_workspace(ws)

    def step(algo_=algo):
        mp.mpgemm(dA, dB, dC, algo_, cutoff)

    for _ in range(a.warmup):
        step()
    mp.check_status("warmup")
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(a.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    clk = clocks.stop()
    mp.check_status("timed")
    barrier()
    ms = allmax(ms)
    value = rep.whole_job(flops, ms * 1e-3) / 1e9

    # kernel-level timing of the same steps (CUDA events around every launch)
    mp.profile_enable(True)
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    prof = mp.profile_read()
    mp.profile_enable(False)
    launches_per_step = sum(v[0] for v in prof.values()) / a.steps
    W32 = (p + 31) // 32
    imad_per_madd = 2 * W32 * W32            # schoolbook: ceil(p/32)^2 partial products, lo + hi
    if algo != 0:
        # the Block leaves: TMA-staged where the layout allows, else thread-staged
        leaf_name = "leaf_tma" if prof["leaf_tma"][0] else "leaf_gemm"
        nl, lms, lunits = (prof["leaf_gemm"][k] + prof["leaf_tma"][k] for k in range(3))
    else:
        leaf_name = "simple_gemm"
        nl, lms, lunits = prof[leaf_name]
    sm_mhz = clk.get("sm_mhz") or 2070.0
    peak = SM_COUNT_GB300 * PEAK_IMAD_PER_CLK_PER_SM * 2070e6 / 1e12      # T IMAD/s at max clock
    achieved = (lunits * imad_per_madd) / (lms * 1e-3) / 1e12 if lms > 0 else 0.0
    # partial products the leaf actually forms: the truncated product keeps the
    # columns i + j >= W - 2 of the W x W schoolbook (2W - 1 + W(W-1)/2 of W^2)
    # when p = 32 W, the case of the configured precisions
    formed = (2 * W32 - 1 + W32 * (W32 - 1) // 2) if 32 * W32 == p else W32 * W32
    kernels = {k: {"launches_per_step": v[0] / a.steps, "ms_per_step": v[1] / a.steps,
                   "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-9)}
               for k, v in prof.items() if v[0]}
    # HBM roofline of the recursion's elementwise kernels: algorithmic bytes
    # = the numbers each launch reads and writes (the library's work units
    # for these classes): operand sums read 4 quadrants and write the 7
    # children, at the last level only the children that are not plain
    # quadrants of the parent (the leaves read those in place);
    # combinations read 7 child products and write 4
    be = 8 * ((p + 63) // 64) + 9
    hbm = measured_peaks().get("hbm_gbs", 6768.4)
    for k in ("operands", "combine"):
        if k in kernels and prof[k][1] > 0:
            gbs = prof[k][2] * be / (prof[k][1] * 1e-3) / 1e9
            kernels[k]["achieved_gbs"] = round(gbs, 1)
            kernels[k]["hbm_frac"] = round(gbs / hbm, 3)

    # end to end through the public API with host buffers (pinned), copies
    # timed: every step copies its A and B in, multiplies and copies C out.
    # Two device buffer sets let one step's copies overlap the neighbouring
    # steps' products (copies on their own streams, ordered by events).
    hA = [t.cpu().pin_memory() for t in (dA.limb, dA.exp, dA.sign)]
    hB = [t.cpu().pin_memory() for t in (dB.limb, dB.exp, dB.sign)]
    hC = [[torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (dC.limb, dC.exp, dC.sign)]
          for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in hA + hB)
    d2h = sum(t.numel() * t.element_size() for t in hC[0])
    bufs = [(dA, dB, dC), (mp.DeviceMP.empty(n, n, p), mp.DeviceMP.empty(n, n, p), mp.DeviceMP.empty(n, n, p))]
    cp_in, cp_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("in", "comp", "out")}
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    cp_in.wait_event(e0)
    e2e_steps = max(1, min(a.steps, 5))
    for s_ in range(e2e_steps):
        bA, bB, bC = bufs[s_ % 2]
        b_ = s_ % 2
        if s_ >= 2:
            cp_in.wait_event(ev["comp"][b_])          # this buffer's last product is done
        with torch.cuda.stream(cp_in):
            for dst, src in zip((bA.limb, bA.exp, bA.sign, bB.limb, bB.exp, bB.sign), hA + hB):
                dst.copy_(src, non_blocking=True)
        ev["in"][b_].record(cp_in)
        stream.wait_event(ev["in"][b_])
        if s_ >= 2:
            stream.wait_event(ev["out"][b_])          # its last result has left
        mp.mpgemm(bA, bB, bC, algo, cutoff)
        ev["comp"][b_].record(stream)
        cp_out.wait_event(ev["comp"][b_])
        with torch.cuda.stream(cp_out):
            for dst, src in zip(hC[b_], (bC.limb, bC.exp, bC.sign)):
                dst.copy_(src, non_blocking=True)
        ev["out"][b_].record(cp_out)
    for b_ in range(min(2, e2e_steps)):
        stream.wait_event(ev["out"][b_])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = allmax(e0.elapsed_time(e1) / e2e_steps)
    mp.check_status("e2e")
    del bufs

    extras, extras_lu, serving, by_prec, split_small, other_configs = {}, None, None, {}, None, None
    serving_repeat = None
    if not a.no_extras and rank == 0 and world == 1:      # the scaling runs report the headline only
        for name in ("simple", "block", "strassen", "winograd"):
            if name == a.algo:
                extras[name] = round(value / world, 3)
                continue
            wsz = mp.workspace_size(n, n, n, p, ALGO_NAMES[name], cutoff)
            if wsz > ws.numel():
                ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
                mp.set_workspace(ws)
            step(ALGO_NAMES[name])
            torch.cuda.synchronize()
            e0.record(stream)
            step(ALGO_NAMES[name])
            e1.record(stream)
            torch.cuda.synchronize()
            extras[name] = round(flops / (e0.elapsed_time(e1) * 1e-3) / 1e9, 3)
        mp.check_status("extras")
        del dA, dB, dC
        mp.set_workspace(None)
        del ws
        torch.cuda.empty_cache()
        # the metric's precisions: Winograd vs Simple at 256 and 1024 bits, same n
        for pp in (256, 1024):
            Ap = mp.DeviceMP.from_host(gen.uniform_pm1(n, n, pp, 33, -16, 16))
            Bp = mp.DeviceMP.from_host(gen.uniform_pm1(n, n, pp, 34, -16, 16))
            Cp = mp.DeviceMP.empty(n, n, pp)
            res = {}
            for name in ("simple", "winograd"):
                mp.mpgemm(Ap, Bp, Cp, ALGO_NAMES[name], cutoff)       # warm (module load)
                torch.cuda.synchronize()
                e0.record(stream)
                mp.mpgemm(Ap, Bp, Cp, ALGO_NAMES[name], cutoff)
                e1.record(stream)
                torch.cuda.synchronize()
                res[name] = round(flops / (e0.elapsed_time(e1) * 1e-3) / 1e9, 3)
            res["speedup_winograd_vs_simple"] = round(res["winograd"] / res["simple"], 3)
            by_prec["p%d" % pp] = res
            mp.check_status("by precision")
            del Ap, Bp, Cp
            torch.cuda.empty_cache()
        extras_lu = [lu_run(a.lu_n, 256, mp.WINOGRAD), lu_run(a.lu_n, 256, mp.SIMPLE),
                     lu_run(a.lu_n, 1024, mp.WINOGRAD),
                     lu_run(a.lu_n, 256, mp.WINOGRAD, kind="lotkin"),
                     lu_run(a.lu_n, 1024, mp.WINOGRAD, kind="lotkin")]
        extras_lu += [lu_run(2 * a.lu_n, p_, mp.WINOGRAD, kind=k_) for k_ in ("well", "lotkin")
                      for p_ in (256, 1024)]
        mp.set_stream(stream)
        other_configs = configs_run(stream)
        mp.set_stream(stream)
        split_small = split_run(4096, 1024, with_simple=False, with_full=False)
        mp.set_stream(stream)
        serving = serve_run(a.serve_requests)
        mp.set_stream(stream)
        serving_repeat = serve_repeat_run()
        mp.set_stream(stream)

    cpu = None
    if rank == 0 and world == 1 and not a.no_extras:
        cpu = cpu_baseline(A, B, a.cpu_seconds, a.cutoff)

    if rank == 0:
        line = {
            "metric": "eff. MP GFLOP/s (2mln/t)",
            "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "mp%d (u32-limb integer)" % p,
            "data": "synthetic", "config": dict(workload_config(a),
                                                leaf_staging="tma" if a.leaf_tma else "threads"),
            "parallelism": "replicas" if world > 1 else "single",
            "roofline": {"bound": "alu", "kernel": "%s (class %s)" % (KERNEL_OF_CLASS[leaf_name], leaf_name),
                         "achieved": round(achieved, 3),
                         "peak": round(peak, 3), "unit": "T IMAD/s",
                         "frac": round(achieved / peak, 4),
                         "peak_note": "derived: 152 SMs x 64 IMAD/clk x 2070 MHz",
                         "work_per_madd_imad": imad_per_madd,
                         "achieved_formed": round(achieved * formed / (W32 * W32), 3),
                         "frac_formed": round(achieved * formed / (W32 * W32) / peak, 4),
                         "formed_note": "IMAD of the %d of %d partial products the truncated product forms"
                                        % (formed, W32 * W32),
                         "traffic": leaf_traffic(a),
                         "traffic_unit": "bytes per launch (ncu capture, scaled by leaves)"},
            "kernels": kernels,
            "gpu_launches": int(round(launches_per_step * a.steps)),
            "e2e": {"value": round(rep.whole_job(flops, e2e_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "copies": "pinned host <-> device every step, overlapping the neighbouring products "
                              "(two device buffer sets, copy streams)"},
            "clocks": clk,
            "algos_gflops": extras,
        }
        if extras.get("simple"):
            line["speedup_vs_simple"] = round(extras.get(a.algo, value) / extras["simple"], 3)
        if cpu:
            line["cpu_baseline"] = cpu
        if by_prec:
            line["by_precision_n%d" % n] = by_prec
        if extras_lu:
            line["lu"] = extras_lu
        if split_small:
            line["split_form_n4096_p1024"] = split_small
        if other_configs:
            line["configs"] = other_configs
        if serving:
            line["serving"] = serving
        if serving_repeat:
            line["serving_repeated_shapes"] = serving_repeat
        print(json.dumps(line), flush=True)
    rep.close()


def _log2abs(M):
    """log2 |x| of every entry of a device MP matrix (-inf for zeros), from
    the top limb and the exponent; no double-range limit on the exponent."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import inputs as gen

    torch.cuda.synchronize()             # the library works on its own stream
    H = M.to_host()
    f = H.limb[0].astype(np.float64) * 2.0 ** -64
    with np.errstate(divide="ignore"):
        out = np.log2(f) + H.exp.astype(np.float64)
    return np.where(H.exp == gen.EXP_ZERO, -np.inf, out)


def configs_run(stream):
    """The other configurations' measurements: the 64^3 Simple product at 256
    bits alone and as a batch of 1024, the 512-bit products at n = 1023 and
    1024, and every algorithm's relative error against the exact product
    rounded to 2p (the library's exact-dot kernel at 2p, which the tests pin
    to the oracle), in units of 2^-p: normwise (max |error| / max |exact|),
    and per output (median and maximum; the maximum comes from outputs whose
    exact value nearly cancels)."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        best = None
        for _ in range(reps):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            best = t if best is None else min(best, t)
        return best

    out = {}
    # configuration 1: Simple 64^3 at 256 bits, alone and 1024 independent ones
    A = mp.DeviceMP.from_host(gen.uniform_pm1(64, 64, 256, 1))
    B = mp.DeviceMP.from_host(gen.uniform_pm1(64, 64, 256, 2))
    C = mp.DeviceMP.empty(64, 64, 256)
    t1 = timed(lambda: mp.mpgemm(A, B, C, mp.SIMPLE))
    Ab = mp.DeviceMP.from_host(gen.uniform_pm1(64 * 1024, 64, 256, 1))
    Bb = mp.DeviceMP.from_host(gen.uniform_pm1(64 * 1024, 64, 256, 2))
    Cb = mp.DeviceMP.empty(64 * 1024, 64, 256)
    tb = timed(lambda: mp.mpgemm_batched(1024, Ab, Bb, Cb, mp.BLOCK))
    out["simple_64_p256"] = {"single_ms": round(t1 * 1e3, 4), "single_gflops": round(2 * 64 ** 3 / t1 / 1e9, 3),
                             "batch1024_ms": round(tb * 1e3, 3),
                             "batch1024_gflops": round(1024 * 2 * 64 ** 3 / tb / 1e9, 3)}
    del A, B, C, Ab, Bb, Cb
    # configuration 2: the odd and the power-of-two size at 512 bits
    sizes = {}
    for n in (1023, 1024):
        A = mp.DeviceMP.from_host(gen.uniform_pm1(n, n, 512, 3, -16, 16))
        B = mp.DeviceMP.from_host(gen.uniform_pm1(n, n, 512, 4, -16, 16))
        C = mp.DeviceMP.empty(n, n, 512)
        res = {}
        for name, algo in ALGO_NAMES.items():
            t = timed(lambda: mp.mpgemm(A, B, C, algo, 64), reps=2)
            res[name] = round(2.0 * n ** 3 / t / 1e9, 3)
        res["speedup_winograd_vs_simple"] = round(res["winograd"] / res["simple"], 3)
        sizes["n%d" % n] = res
        del A, B, C
    out["p512_sizes"] = sizes
    # relative errors against the exact product rounded to 2p, n = 512
    errs = {}
    n = 512
    for p in (128, 512, 1024):
        A = mp.DeviceMP.from_host(gen.uniform_pm1(n, n, p, 21, -16, 16))
        B = mp.DeviceMP.from_host(gen.uniform_pm1(n, n, p, 22, -16, 16))
        A2, B2 = mp.DeviceMP.empty(n, n, 2 * p), mp.DeviceMP.empty(n, n, 2 * p)
        mp.convert(A, A2)
        mp.convert(B, B2)
        ref = mp.DeviceMP.empty(n, n, 2 * p)
        mp.mpgemm(A2, B2, ref, mp.EXACT)
        lref = _log2abs(ref)
        res = {}
        for name, algo in ALGO_NAMES.items():
            C = mp.DeviceMP.empty(n, n, p)
            mp.mpgemm(A, B, C, algo, 64)
            C2 = mp.DeviceMP.empty(n, n, 2 * p)
            mp.convert(C, C2)
            D = mp.DeviceMP.empty(n, n, 2 * p)
            mp.elementwise(mp.OP_SUB, C2, ref, D)
            ld = _log2abs(D)
            ok = np.isfinite(lref)
            rel = (ld - lref + p)[ok]                    # log2 of |error| / |exact| in units of 2^-p
            # normwise: max |error| / max |exact|; componentwise: median and max
            res[name] = {"normwise_ulp": float(2.0 ** (ld.max() - lref[ok].max() + p)) if np.isfinite(ld.max()) else 0.0,
                         "median_ulp": float(2.0 ** np.median(rel)),
                         "max_componentwise_ulp": float(2.0 ** min(rel.max(), 1000.0)),
                         "exact_outputs": int(np.sum(~np.isfinite(ld)))}
            del C, C2, D
        errs["p%d" % p] = res
        mp.check_status("errors")
        del A, B, A2, B2, ref
    out["rel_error_vs_exact_2p_n512"] = errs
    torch.cuda.empty_cache()
    return out


def lu_run(n, p, algo, panel=128, cutoff=64, kind="well"):
    """One MP LU solve of A x = b, b = A * ones (Simple product), on the GPU:
    seconds, and the backward / forward errors computed by the library at 2p."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    A = gen.well_conditioned(n, p, 5) if kind == "well" else gen.lotkin(n, p)
    dA = mp.DeviceMP.from_host(A)
    dA0 = mp.DeviceMP.from_host(A)
    ones = mp.DeviceMP.from_host(gen.ones(n, 1, p))
    db = mp.DeviceMP.empty(n, 1, p)
    mp.mpgemm(dA0, ones, db, mp.SIMPLE)
    dx = mp.DeviceMP.empty(n, 1, p)
    piv = torch.zeros(n, dtype=torch.int64, device="cuda")
    mp.set_lu(panel, algo, cutoff)
    torch.cuda.synchronize()
    # timed without per-launch events; a second factorisation of a fresh copy
    # of A, with the library's per-launch CUDA events, gives the kernel shares
    t0 = time.perf_counter()
    mp.mplu(dA, piv, db, dx)
    rc = mp.sync_status()
    t = time.perf_counter() - t0
    dA2 = mp.DeviceMP.from_host(A)
    dx2 = mp.DeviceMP.empty(n, 1, p)
    torch.cuda.synchronize()
    mp.profile_enable(True)
    mp.mplu(dA2, piv, db, dx2)
    mp.check_status("profiled LU")
    prof = mp.profile_read()
    mp.profile_enable(False)
    del dA2, dx2
    mp.set_lu(128, mp.SIMPLE, 64)
    # residual r = b - A x at 2p (exact widening, Simple product, one subtraction)
    q = 2 * p
    wA, wx, wb = (mp.DeviceMP.empty(r, c, q) for r, c in ((n, n), (n, 1), (n, 1)))
    mp.convert(dA0, wA)
    mp.convert(dx, wx)
    mp.convert(db, wb)
    Ax = mp.DeviceMP.empty(n, 1, q)
    mp.mpgemm(wA, wx, Ax, mp.SIMPLE)
    r = mp.DeviceMP.empty(n, 1, q)
    mp.elementwise(mp.OP_SUB, wb, Ax, r)
    one = mp.DeviceMP.from_host(gen.ones(n, 1, q))
    fe = mp.DeviceMP.empty(n, 1, q)
    mp.elementwise(mp.OP_SUB, wx, one, fe)
    mp.check_status("lu residual")

    # norms in log2 space: the residual and the error of x sit near 2^-p,
    # below the double range at 1024 bits and above
    la = _log2abs(dA0)
    rowmax = la.max(axis=1, keepdims=True)
    rowmax = np.where(np.isfinite(rowmax), rowmax, 0.0)
    l_anorm = float((rowmax[:, 0] + np.log2(np.exp2(la - rowmax).sum(axis=1))).max())
    l_xn, l_bn = float(_log2abs(dx).max()), float(_log2abs(db).max())
    hi = max(l_anorm + l_xn, l_bn)
    l_den = hi + np.log2(np.exp2(l_anorm + l_xn - hi) + np.exp2(l_bn - hi))
    l_back = float(_log2abs(r).max()) - l_den
    l_fwd = float(_log2abs(fe).max())
    back, fwd = float(2.0 ** l_back), float(2.0 ** l_fwd)
    dev_ms = sum(v[1] for v in prof.values())
    # the trailing products' leaves against the derived integer peak: one
    # multiply-add is 2 ceil(p/32)^2 IMAD of schoolbook partial products
    leaf_n, leaf_ms, leaf_madds = (prof["leaf_gemm"][k] + prof["leaf_tma"][k] for k in range(3))
    leaf_roof = None
    if leaf_n and leaf_ms > 0:
        wds = -(-p // 32)
        ach = leaf_madds * 2 * wds * wds / (leaf_ms * 1e-3) / 1e12
        leaf_roof = {"bound": "alu", "achieved": round(ach, 3), "peak": 20.137, "unit": "T IMAD/s",
                     "frac": round(ach / 20.137, 4), "work_per_madd_imad": 2 * wds * wds,
                     "peak_note": "derived: 152 SMs x 64 IMAD/clk x 2070 MHz"}
    return {"n": n, "prec": p, "algo": {0: "simple", 1: "block", 2: "strassen", 3: "winograd"}[algo],
            "panel": panel, "matrix": kind, "seconds": round(t, 4), "status": rc,
            "kernel_ms": {k: round(v[1], 2) for k, v in prof.items() if v[0]},
            "kernel_share": {k: round(v[1] / dev_ms, 4) for k, v in prof.items() if v[0] and dev_ms > 0},
            "trailing_leaf_roofline": leaf_roof,
            "launches": int(sum(v[0] for v in prof.values())),
            "eff_gflops": round((2.0 / 3.0) * n ** 3 / t / 1e9, 4),
            "backward_error": back, "forward_error": fwd,
            "backward_error_log10": round(l_back * math.log10(2.0), 2),
            "forward_error_log10": round(l_fwd * math.log10(2.0), 2)}


def lu_sweep_run(n=1024, precs=(256, 1024), algos=(0, 2, 3), alphas=range(1, 11), seed=21,
                 kind="random", runs_for=None):
    """The paper's LU experiment (Sec. 4): no pivoting, a random matrix with
    entries in [-1, 1) (seeded) or the Lotkin matrix, x = [0, 1, ..., n-1],
    b = A x (Simple product at p), block size K = alpha * 32 for
    alpha = 1..10, the trailing update by Simple, Strassen or Winograd
    (n_min = 32); plus the column-wise LU (one panel of n columns, no
    trailing product) as the baseline.  runs_for(p) may replace the run list
    of a precision.  Per run: seconds and the maximum relative error
    max_i |x~_i - i| / i over i >= 1 (x~_0 enters as |x~_0|), the
    difference taken at 2p (exact widening) or, above 4352 bits, at p
    (exact by Sterbenz's lemma while x~_i is within a factor 2 of i)."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    names = {0: "simple", 1: "block", 2: "strassen", 3: "winograd"}
    out = []
    mp.set_lu_pivoting(False)
    try:
        for p in precs:
            A = gen.uniform_pm1(n, n, p, seed) if kind == "random" else gen.lotkin(n, p)
            dA0 = mp.DeviceMP.from_host(A)
            dxt = mp.DeviceMP.from_host(gen.from_ints([[i] for i in range(n)], p))
            db = mp.DeviceMP.empty(n, 1, p)
            mp.mpgemm(dA0, dxt, db, mp.SIMPLE)
            q = 2 * p if 2 * p <= 8704 else p
            wxt = mp.DeviceMP.from_host(gen.from_ints([[i] for i in range(n)], q))
            runs = [("columnwise", mp.SIMPLE, n)] + [(names[a], a, 32 * al) for a in algos for al in alphas]
            if runs_for is not None:
                runs = runs_for(p)
            for name, algo, K in runs:
                dA = mp.DeviceMP.empty(n, n, p)
                dA.limb.copy_(dA0.limb)
                dA.exp.copy_(dA0.exp)
                dA.sign.copy_(dA0.sign)
                dx = mp.DeviceMP.empty(n, 1, p)
                piv = torch.zeros(n, dtype=torch.int64, device="cuda")
                mp.set_lu(K, algo, 32)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                mp.mplu(dA, piv, db, dx)
                rc = mp.sync_status()
                t = time.perf_counter() - t0
                wx = mp.DeviceMP.empty(n, 1, q)
                mp.convert(dx, wx)
                fe = mp.DeviceMP.empty(n, 1, q)
                mp.elementwise(mp.OP_SUB, wx, wxt, fe)
                mp.check_status("forward error")
                torch.cuda.synchronize()
                H = fe.to_host()
                lg = np.log2(np.maximum(H.limb[0].astype(np.float64), 1.0) * 2.0 ** -64) + \
                    np.where(H.exp == gen.EXP_ZERO, -np.inf, H.exp.astype(np.float64))
                rel = lg[:, 0] - np.log2(np.maximum(np.arange(n), 1))
                mx = float(np.max(rel))
                out.append({"prec": p, "update": name, "K": K, "alpha": K // 32 if name != "columnwise" else None,
                            "seconds": round(t, 4), "status": rc,
                            "max_rel_err_log10": round(mx * np.log10(2.0), 2) if np.isfinite(mx) else None})
    finally:
        mp.set_lu(128, mp.SIMPLE, 64)
        mp.set_lu_pivoting(True)
    return {"n": n, "matrix": ("uniform [-1,1)" if kind == "random" else "Lotkin") + ", no pivoting",
            "x_true": "0..n-1", "runs": out}


def lotkin_run(n=1024, alphas=(1, 2, 4, 8)):
    """The paper's ill-conditioned case (Sec. 4, its Figure 2): the Lotkin
    matrix without pivoting at 8192 bits (column-wise LU and Winograd
    updates) and at 8650 bits (Winograd updates, the precision the paper
    adds to recover the 138 digits Winograd loses)."""
    def runs_for(p):
        r = [("winograd", 3, 32 * a) for a in alphas]
        return ([("columnwise", 0, n)] + r) if p == 8192 else r
    return lu_sweep_run(n, precs=(8192, 8650), kind="lotkin", runs_for=runs_for)


def cond_run(n=1024, p=5376, panel=128):
    """cond_1 = ||A||_1 ||A^-1||_1 of the n x n Lotkin matrix (Sec. 4 quotes
    4.3e1576 for n = 1024): A^-1 on the GPU at p bits (mplu with partial
    pivoting and Winograd trailing products, then mplu_solve with B = I, the
    272-word wide class above 2048 bits), the 1-norms read in log2 space.
    p must exceed log2 cond_1 (about 5237 bits) for A^-1 to carry correct
    leading digits; 5376 leaves about 40 digits."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen
    from paper_1410_1599_gb300 import norms

    t0 = time.perf_counter()
    A = gen.lotkin(n, p)
    t_gen = time.perf_counter() - t0
    dA = mp.DeviceMP.from_host(A)
    piv = torch.zeros(n, dtype=torch.int64, device="cuda")
    mp.set_lu(panel, mp.WINOGRAD, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mp.mplu(dA, piv, None, None)
    rc_lu = mp.sync_status()
    t_lu = time.perf_counter() - t0
    mp.set_lu(128, mp.SIMPLE, 64)
    dI = mp.DeviceMP.from_host(gen.identity(n, p))
    dX = mp.DeviceMP.empty(n, n, p)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mp.mplu_solve(dA, piv, dI, dX)
    rc_inv = mp.sync_status()
    t_inv = time.perf_counter() - t0
    X = dX.to_host()
    la, lx = norms.norm1_log2(A), norms.norm1_log2(X)
    l10 = norms.log10_of_log2(la + lx)
    mant = 10 ** (l10 - math.floor(l10))
    exact = None                            # the oracle's exact value, stored by tests/golden/make_lotkin_cond1.py
    gold = os.path.join(ROOT, "tests", "golden", "lotkin_cond1.txt")
    if os.path.exists(gold):
        for ln in open(gold):
            f = ln.split()
            if f and not ln.startswith("#") and int(f[0]) == n:
                exact = float(f[3])
    return {"n": n, "prec": p, "matrix": "lotkin", "panel": panel, "status_lu": rc_lu, "status_inverse": rc_inv,
            "seconds_lu": round(t_lu, 2), "seconds_inverse": round(t_inv, 2), "seconds_host_generation": round(t_gen, 1),
            "norm1_A": round(2.0 ** la, 6), "log10_norm1_inverse": round(norms.log10_of_log2(lx), 3),
            "cond1": "%.3fe%d" % (mant, math.floor(l10)), "log10_cond1": round(l10, 4),
            "log10_cond1_exact": exact,
            "paper_cond1": "4.3e1576 (Sec. 4, n = 1024)"}


def serve_run(n_req, seed=11, slots=8, budget=150 << 30):
    """Config-5 style request stream through the library's serving loop:
    70% GEMM (m, l, n ~ U{16..2048}), 30% LU solve (n ~ U{64..1024}),
    precision ~ U{128, 256, 512, 1024, 2048}; operands are tiles of per-precision
    pools of seeded U[-1,1)*2^e entries.  Phase 1 submits everything at once
    (capacity, requests/s); phase 2 replays a Poisson stream at 0.7 x capacity
    and reports latency percentiles."""
    import numpy as np

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    rng = np.random.default_rng(seed)
    precs = [128, 256, 512, 1024, 2048]
    pool = {p: gen.uniform_pm1(512, 512, p, 77 + p, -16, 16) for p in precs}

    def tile(p, rows, cols, off):
        P = pool[p]
        ri = (np.arange(rows) + off) % 512
        ci = (np.arange(cols) + 3 * off) % 512
        return P.sub(ri, ci)

    specs = []
    for i in range(n_req):
        p = int(rng.choice(precs))
        if rng.random() < 0.7:
            m, l, n = (int(x) for x in rng.integers(16, 2049, 3))
            algo = mp.WINOGRAD if min(m, l, n) > 128 else mp.BLOCK
            specs.append(("gemm", i, p, (m, l, n), algo, int(rng.integers(0, 512))))
        else:
            n = int(rng.integers(64, 1025))
            specs.append(("lu", i, p, (n,), mp.WINOGRAD if n > 256 else mp.SIMPLE, int(rng.integers(0, 512))))

    def make(spec):
        kind, i, p, dims, algo, off = spec
        if kind == "gemm":
            m, l, n = dims
            return tile(p, m, l, off), tile(p, l, n, off + 7)
        n = dims[0]
        A = tile(p, n, n, off)
        q = p - n.bit_length() - 2          # diagonal n + v exact in p bits (as well_conditioned)
        D = gen.from_exact_ints([((n << q) + k < 0, abs((n << q) + k), q) for k in
                                 (gen.rand_bits(seed + i, j, q + 1) - (1 << q) for j in range(n))], p, (1, n))
        for j in range(n):
            A.limb[:, j, j] = D.limb[:, 0, j]
            A.exp[j, j] = D.exp[0, j]
            A.sign[j, j] = D.sign[0, j]
        return A, tile(p, n, 1, off + 11)

    flops = [2.0 * s[3][0] * s[3][1] * s[3][2] if s[0] == "gemm" else (2.0 / 3.0) * s[3][0] ** 3
             for s in specs]

    def prepare(srv, s):
        kind, i, p, dims, algo, off = s
        X, Y = make(s)
        if kind == "gemm":
            return srv.prepare_gemm(i, X, Y, algo=algo, cutoff=64)
        return srv.prepare_lu(i, X, Y, algo=algo, cutoff=64, panel=128)

    # Requests are prepared (operands tiled and copied into page-locked host
    # buffers) ahead of their submission by a helper thread, at most `window`
    # of them at a time, so that submitting only queues a request; outputs of
    # long runs are not kept (their status and latency are).
    import queue as queue_mod
    import threading

    window = max(48, slots * 6) if n_req > 64 else n_req

    def ahead(srv):
        q = queue_mod.Queue(maxsize=window)

        def work():
            for s in specs:
                q.put(prepare(srv, s))
        th = threading.Thread(target=work, daemon=True)
        th.start()
        return q, th

    keep = n_req <= 64
    # phase 1: closed loop (the preparation window fills before the clock
    # starts).  Up to `window` requests are outstanding at once: all of them
    # for the default 32-request stream, a sliding window for long streams
    # (whose pinned host buffers would not all fit in host memory).
    srv = mp.Server(budget_bytes=budget, slots=slots, keep_outputs=keep)
    q, th = ahead(srv)
    while q.qsize() < min(window, n_req) and th.is_alive():
        time.sleep(0.01)
    t0 = time.perf_counter()
    submitted = finished = 0
    while finished < n_req:
        while submitted < n_req and submitted - finished < window:
            assert srv.submit(q.get()) == 0
            submitted += 1
        finished += len(srv.poll())
        if finished < n_req:
            time.sleep(0.001)
    srv.drain()
    t_cap = time.perf_counter() - t0
    th.join()
    st1 = srv.stats()
    srv.close()
    cap = n_req / t_cap
    # phase 2: Poisson arrivals at 0.7 x capacity
    lam = 0.7 * cap
    gaps = rng.exponential(1.0 / lam, n_req)
    srv = mp.Server(budget_bytes=budget, slots=slots, keep_outputs=keep)
    q, th = ahead(srv)
    while q.qsize() < min(window, n_req) and th.is_alive():
        time.sleep(0.01)
    t0 = time.perf_counter()
    due = t0
    for g in gaps:
        due += g
        while time.perf_counter() < due:
            time.sleep(min(0.002, max(0.0, due - time.perf_counter())))
            srv.poll()                      # finished requests release their host buffers
        assert srv.submit(q.get()) == 0
    srv.drain()
    t_run = time.perf_counter() - t0
    st2 = srv.stats()
    lat = np.array([srv.results[i][1] for i in range(n_req)])
    ok = all(srv.results[i][0] == mp.REQ_DONE for i in range(n_req))
    srv.close()
    return {"requests": n_req, "mix": "70% GEMM m,l,n~U{16..2048}, 30% LU n~U{64..1024}, p~U{128..2048}",
            "slots": slots, "budget_gb": budget / 2 ** 30, "all_done": ok,
            "capacity_req_per_s": round(cap, 3), "offered_req_per_s": round(lam, 3),
            "throughput_req_per_s": round(n_req / t_run, 3),
            "eff_gflops_closed_loop": round(sum(flops) / t_cap / 1e9, 3),
            "p50_ms": round(float(np.percentile(lat, 50)), 2),
            "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "batches": st1["batches"], "batched_requests": st1["batched_requests"],
            "batches_poisson": st2["batches"], "batched_requests_poisson": st2["batched_requests"],
            "peak_gb": round(max(st1["peak_bytes"], st2["peak_bytes"]) / 2 ** 30, 3)}


def serve_repeat_run(n_req=96, seed=12, slots=8, budget=150 << 30):
    """Requests drawn from eight fixed shapes (four GEMMs, four LU solves,
    256 and 512 bits), each with its own data, through the serving loop with
    the CUDA-graph cache off and on: closed-loop capacity, then Poisson
    arrivals at 0.7 x the cache-off capacity, p50 / p99 latency."""
    import numpy as np

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    rng = np.random.default_rng(seed)
    shapes = [("gemm", 256, (96, 96, 96), mp.BLOCK), ("gemm", 512, (200, 160, 180), mp.WINOGRAD),
              ("gemm", 256, (384, 384, 384), mp.WINOGRAD), ("gemm", 512, (64, 512, 64), mp.BLOCK),
              ("lu", 256, (128,), mp.SIMPLE), ("lu", 512, (96,), mp.SIMPLE),
              ("lu", 256, (320,), mp.WINOGRAD), ("lu", 512, (200,), mp.SIMPLE)]
    picks = rng.integers(0, len(shapes), n_req)
    inputs = []
    for i, k in enumerate(picks):
        kind, p, dims, algo = shapes[k]
        if kind == "gemm":
            m, l, n = dims
            inputs.append((kind, p, algo, gen.uniform_pm1(m, l, p, 9000 + i, -16, 16),
                           gen.uniform_pm1(l, n, p, 19000 + i, -16, 16)))
        else:
            n = dims[0]
            inputs.append((kind, p, algo, gen.well_conditioned(n, p, 29000 + i), gen.uniform_pm1(n, 1, p, 39000 + i)))

    def submit(srv, i):
        kind, p, algo, X, Y = inputs[i]
        if kind == "gemm":
            return srv.submit_gemm(i, X, Y, algo=algo, cutoff=64)
        return srv.submit_lu(i, X, Y, algo=algo, cutoff=64, panel=128)

    res = {}
    lam = None
    for graphs in (0, 8):
        srv = mp.Server(budget_bytes=budget, slots=slots)
        srv.set_graphs(graphs)
        t0 = time.perf_counter()
        for i in range(n_req):
            assert submit(srv, i) == 0
        srv.drain()
        cap = n_req / (time.perf_counter() - t0)
        g1 = srv.graph_stats()
        srv.close()
        if lam is None:
            lam = 0.7 * cap
        gaps = np.random.default_rng(seed + 1).exponential(1.0 / lam, n_req)
        srv = mp.Server(budget_bytes=budget, slots=slots)
        srv.set_graphs(graphs)
        t0 = time.perf_counter()
        due = t0
        for i, g in enumerate(gaps):
            due += g
            while time.perf_counter() < due:
                time.sleep(min(0.002, max(0.0, due - time.perf_counter())))
            assert submit(srv, i) == 0
        srv.drain()
        lat = np.array([srv.results[i][1] for i in range(n_req)])
        ok = all(srv.results[i][0] == mp.REQ_DONE for i in range(n_req))
        g2 = srv.graph_stats()
        srv.close()
        res["graphs_%s" % ("on" if graphs else "off")] = {
            "all_done": ok, "capacity_req_per_s": round(cap, 2), "p50_ms": round(float(np.percentile(lat, 50)), 2),
            "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "graph_replays": g1["replays"] + g2["replays"], "graphs_captured": g1["captured"] + g2["captured"]}
    return {"requests": n_req, "shapes": len(shapes), "offered_req_per_s": round(lam, 2), **res}


def split_run(n=4096, p=1024, with_simple=True, exp_lo=-16, exp_hi=16, with_exact=True, with_full=True):
    """Split form vs the exact limb path (same correctly rounded result) on
    n^3 at p bits, entries U[-1,1)*2^e, e ~ U{-16..16}: the truncated split
    form (default), the full split form (every digit diagonal), the exact
    limb kernel and, for scale, the per-operation-rounded Simple kernel."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    A = gen.uniform_pm1(n, n, p, 13, exp_lo, exp_hi)
    B = gen.uniform_pm1(n, n, p, 14, exp_lo, exp_hi)
    dA, dB = mp.DeviceMP.from_host(A), mp.DeviceMP.from_host(B)
    out = {}
    res = {}
    runs = (("split", mp.SPLIT, True),) + ((("split_full", mp.SPLIT, False),) if with_full else ()) + \
        ((("exact_limb", mp.EXACT, True),) if with_exact else ()) + \
        ((("simple_limb", mp.SIMPLE, True),) if with_simple else ())
    for name, algo, trunc in runs:
        C = mp.DeviceMP.empty(n, n, p)
        mp.set_split_truncation(trunc)
        torch.cuda.synchronize()
        mp.profile_enable(True)
        t0 = time.perf_counter()
        mp.mpgemm(dA, dB, C, algo, 64)
        rc = mp.sync_status()
        t = time.perf_counter() - t0
        prof = mp.profile_read()
        mp.profile_enable(False)
        mp.set_split_truncation(True)
        out[name] = {"seconds": round(t, 3), "eff_gflops": round(2.0 * n ** 3 / t / 1e9, 3), "status": rc,
                     "kernels_ms": {k: round(v[1], 2) for k, v in prof.items() if v[0]}}
        if algo == mp.SPLIT:
            S = (p + 64 + 7) // 8 + 1
            macs = prof["split_slices"][2]
            out[name]["digits"] = S
            out[name]["digit_pairs_kept"] = round(macs / (S * S * n * float(-(-n // 32) * 32) * n), 4)
            out[name]["exact_fallback_outputs"] = mp.split_fallbacks()
            out[name]["tensor_macs"] = macs
            tflops = 2.0 * macs / (prof["split_slices"][1] * 1e-3) / 1e12
            out[name]["slice_tmac_per_s"] = round(tflops / 2.0, 2)
            # fp16 inputs, fp32 accumulation: the same tensor rate as bf16
            peak = measured_peaks().get("bf16_tflops", 1900.0)
            out[name]["roofline"] = {"bound": "tensor", "kernel": "split_slice_tc_kernel (tcgen05 kind::f16)",
                                     "achieved": round(tflops, 1), "peak": peak, "unit": "TFLOP/s",
                                     "frac": round(tflops / peak, 4),
                                     "peak_note": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"}
        res[name] = C
    def equal(X, Y):
        return bool(torch.equal(X.limb, Y.limb) and torch.equal(X.exp, Y.exp) and torch.equal(X.sign, Y.sign))

    ref = res["exact_limb"] if with_exact else res["split_full"]
    same = equal(res["split"], ref) and (not with_full or equal(res["split_full"], ref))
    wide_rows = int(sum(1 for i in range(n) if (A.exp[i][A.exp[i] != gen.EXP_ZERO]).min()
                        < (A.exp[i][A.exp[i] != gen.EXP_ZERO]).max() - 64))
    wide_cols = int(sum(1 for j in range(n) if (B.exp[:, j][B.exp[:, j] != gen.EXP_ZERO]).min()
                        < (B.exp[:, j][B.exp[:, j] != gen.EXP_ZERO]).max() - 64))
    line = {"n": n, "prec": p, "entries": "U[-1,1)*2^e, e~U{%d..%d}" % (exp_lo, exp_hi),
            ("split_equals_exact_limb_all_outputs" if with_exact else "split_equals_full_split_all_outputs"): same,
            "wide_rows": wide_rows, "wide_cols": wide_cols}
    if with_exact:
        line["speedup_split_vs_exact_limb"] = round(out["exact_limb"]["seconds"] / out["split"]["seconds"], 3)
    return {**line, **out}


# The paper's CPU times (seconds, MPFR on one core of a Core i7 3850; context
# only): Tables 3 and 4 (square n, n_min = 32: min(Simple, Block), Strassen,
# Winograd) and Table 5 (m = n = 1024, varying l: Simple, Block(32),
# Strassen, Winograd).
PAPER_SQUARE = {
    128: {255: (1.06, 0.72, 0.63), 256: (1.22, 0.70, 0.57), 257: (1.04, 0.74, 0.60),
          511: (9.60, 4.84, 4.06), 512: (9.68, 4.77, 3.73), 513: (9.89, 4.92, 3.88),
          1023: (77.63, 32.02, 25.57), 1024: (77.72, 31.53, 24.10), 1025: (78.41, 32.21, 24.77),
          2047: (619.21, 211.80, 163.87), 2048: (618.87, 211.19, 155.67), 2049: (623.24, 212.79, 157.52)},
    1024: {255: (5.46, 2.33, 1.95), 256: (5.53, 2.31, 1.72), 257: (5.61, 2.41, 1.81),
           511: (43.81, 13.40, 10.57), 512: (44.20, 13.02, 9.44), 513: (44.37, 13.38, 9.81),
           1023: (352.79, 76.93, 57.98), 1024: (355.99, 74.58, 52.47), 1025: (356.58, 76.36, 54.22),
           2047: (2820.16, 454.02, 329.41), 2048: (2824.34, 446.87, 302.56), 2049: (2829.95, 456.08, 307.05)},
}
PAPER_RECT = {
    128: {63: (5.09, 5.86, 5.31, 4.29), 64: (5.18, 5.91, 5.03, 3.99), 65: (5.26, 6.30, 5.24, 4.21),
          127: (10.47, 11.8, 9.43, 6.45), 128: (10.54, 11.86, 8.71, 5.42), 129: (10.63, 12.24, 8.90, 5.65),
          255: (52.51, 23.69, 14.67, 9.39), 256: (52.27, 23.77, 13.13, 7.51), 257: (52.56, 24.07, 13.39, 7.70),
          511: (110.75, 47.42, 26.40, 16.55), 512: (106.19, 47.44, 21.85, 11.83), 513: (110.82, 47.96, 22.08, 12.09)},
    1024: {63: (24.71, 26.74, 19.92, 14.88), 64: (25.77, 27.13, 19.49, 14.31), 65: (26.24, 27.82, 20.04, 14.91),
           127: (52.37, 53.75, 32.26, 19.02), 128: (53.17, 54.23, 30.69, 16.74), 129: (53.59, 54.97, 30.79, 17.37),
           255: (105.04, 108.90, 47.43, 24.15), 256: (106.34, 108.64, 43.12, 19.83), 257: (106.92, 109.83, 43.63, 20.48),
           511: (244.07, 216.82, 71.30, 34.18), 512: (245.69, 216.65, 61.01, 25.22), 513: (247.96, 217.69, 62.14, 25.91)},
}


def paper_run(stream, precs=(128, 1024), square=True, rect=True):
    """The paper's Section 4 benchmark on the GPU: a_ij = sqrt(5)(i+j-1),
    b_ij = sqrt(3)(n-i+1); square n in 255..2049 (Tables 2-4) and
    1024 x l x 1024 (Table 5); Simple, Block, Strassen and Winograd with
    n_min = 32 and the mixed odd-size policy (Table 1's counts).  Per run:
    device seconds and the maximum and minimum relative error against the
    exact product, whose rows are taken from the library's exact-dot kernel
    at 2p on the same matrices generated at 2p bits (their own error is
    about 2^-2p, far below the products' 2^-p)."""
    import numpy as np
    import torch

    from paper_1410_1599_gb300 import binding as mp
    from paper_1410_1599_gb300 import inputs as gen

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    algos = (("simple", mp.SIMPLE), ("block", mp.BLOCK), ("strassen", mp.STRASSEN), ("winograd", mp.WINOGRAD))
    mp.set_odd_policy(mp.MIXED)

    def reference_rows(m, l, n, q):
        A2, B2 = gen.sqrt_matrices(m, l, n, q, b_cols=1)    # the columns of B are all alike
        dA2, dB2 = mp.DeviceMP.from_host(A2), mp.DeviceMP.from_host(B2)
        R = mp.DeviceMP.empty(m, 1, q)
        mp.mpgemm(dA2, dB2, R, mp.EXACT, 64)
        mp.check_status("reference rows")
        return R

    def rel_errors(C, R):
        m, n, q = C.rows, C.cols, R.p
        torch.cuda.synchronize()            # R and C come from the library's stream
        C2 = mp.DeviceMP.empty(m, n, q)
        mp.convert(C, C2)
        Rf = mp.DeviceMP(R.limb.expand(-1, -1, n).contiguous(), R.exp.expand(-1, n).contiguous(),
                         R.sign.expand(-1, n).contiguous(), q, m, n)
        torch.cuda.synchronize()            # the expansion ran on torch's stream
        D = mp.DeviceMP.empty(m, n, q)
        mp.elementwise(mp.OP_SUB, C2, Rf, D)
        mp.check_status("error difference")
        torch.cuda.synchronize()
        top = D.limb[0].cpu().numpy().view(np.uint64).astype(np.float64) * 2.0 ** -64
        e = D.exp.cpu().numpy()
        rtop = R.limb[0, :, 0].cpu().numpy().view(np.uint64).astype(np.float64) * 2.0 ** -64
        re = R.exp[:, 0].cpu().numpy().astype(np.float64)
        zero = e == gen.EXP_ZERO
        lg = np.log2(np.where(zero, 1.0, top)) + np.where(zero, 0, e) - (np.log2(rtop) + re)[:, None]
        err = np.where(zero, 0.0, np.exp2(lg))
        return float(err.max()), float(err.min())

    def one(m, l, n, p):
        A, B = gen.sqrt_matrices(m, l, n, p)
        dA, dB = mp.DeviceMP.from_host(A), mp.DeviceMP.from_host(B)
        R = reference_rows(m, l, n, 2 * p)
        row = {"m": m, "l": l, "n": n, "prec": p}
        for name, algo in algos:
            C = mp.DeviceMP.empty(m, n, p)
            mp.mpgemm(dA, dB, C, algo, 32)                 # warm-up
            torch.cuda.synchronize()
            e0.record(stream)
            mp.mpgemm(dA, dB, C, algo, 32)
            e1.record(stream)
            torch.cuda.synchronize()
            rc = mp.sync_status()
            t = e0.elapsed_time(e1) * 1e-3
            mx, mn = rel_errors(C, R)
            row[name] = {"seconds": round(t, 5), "eff_gflops": round(2.0 * m * l * n / t / 1e9, 3),
                         "max_rel_err": mx, "min_rel_err": mn, "status": rc}
        return row

    out = {"square": [], "rectangle": []}
    try:
        for p in precs:
            if square:
                for n in sorted(PAPER_SQUARE[p]):
                    r = one(n, n, n, p)
                    r["paper_cpu_seconds"] = dict(zip(("min_simple_block", "strassen", "winograd"),
                                                      PAPER_SQUARE[p][n]))
                    out["square"].append(r)
            if rect:
                for l in sorted(PAPER_RECT[p]):
                    r = one(1024, l, 1024, p)
                    r["paper_cpu_seconds"] = dict(zip(("simple", "block32", "strassen", "winograd"),
                                                      PAPER_RECT[p][l]))
                    out["rectangle"].append(r)
    finally:
        mp.set_odd_policy(mp.PEEL)
    return out


def winograd_subproduct(A, B, cutoff, levels=2):
    """The oracle (plain C, all host threads) running the same algorithm as
    the GPU line on a bounded part of the same product: Winograd's recursion
    on one node `levels` levels down, i.e. an (n/2^levels)^3 product with the
    same cutoff, precision and odd-size policy (for n = 2048: a 512^3 product,
    one of the 49 level-2 sub-products; the recursion below it is the one the
    full product runs, and the additions of the two levels above it are about
    1 % of the work).  Its operands are the corresponding blocks of A and B.
    Returns (seconds, sub-product size, eff. GFLOP/s of the whole product at
    7^levels sub-products of that time)."""
    import numpy as np

    from oracle import oracle as orc

    n = A.shape[0]
    h = n >> levels
    Asub, Bsub = A.sub(np.arange(h), np.arange(h)), B.sub(np.arange(h), np.arange(h))
    t0 = time.perf_counter()
    orc.gemm(orc.WINOGRAD, Asub, Bsub, cutoff=cutoff)
    t = time.perf_counter() - t0
    return t, h, 2.0 * n ** 3 / (7 ** levels * t) / 1e9


def cpu_baseline(A, B, seconds, cutoff=64):
    """The oracle timed on the host cores, two ways.  value: the same
    algorithm as the GPU line (Winograd, see winograd_subproduct).
    simple_dot_sample: a sample of outputs of the same product by Simple dot
    products, eff GFLOP/s = 2 l outputs / t; the sample (rows x columns of C)
    grows until it takes about `seconds`; only the sampled rows of A and
    columns of B are handed over."""
    import numpy as np

    from oracle import oracle as orc

    tw, h, vw = winograd_subproduct(A, B, cutoff)
    n, l = A.shape
    ncols = B.shape[1]
    threads = orc.max_threads()
    rng = np.random.default_rng(0)

    def run(count):
        r = min(n, count)
        c = min(ncols, max(1, -(-count // r)))
        rows = np.sort(rng.choice(n, size=r, replace=False))
        cols = np.sort(rng.choice(ncols, size=c, replace=False))
        Asub, Bsub = A.sub(rows, np.arange(l)), B.sub(np.arange(l), cols)
        t0 = time.perf_counter()
        orc.gemm(orc.SIMPLE, Asub, Bsub)
        return time.perf_counter() - t0, r, c

    count = threads
    t, r, c = run(count)
    while t < seconds / 8 and r * c < n * ncols:
        count = min(n * ncols, count * 4)
        t, r, c = run(count)
    count = int(max(threads, min(n * ncols, r * c * seconds / max(t, 1e-9))))
    t, r, c = run(count)
    return {"value": round(vw, 6), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
            "sample": "Winograd (cutoff %d) on one of the 49 level-2 sub-products, a %d^3 product "
                      "taking %.2f s on %d threads; whole-product rate = 2 n^3 / (49 t)"
                      % (cutoff, h, tw, threads),
            "seconds": round(tw, 2),
            "simple_dot_sample": {"value": round(2.0 * l * r * c / t / 1e9, 6), "unit": "GFLOP/s",
                                  "sample": "%d x %d outputs of C by Simple dot products (l=%d)" % (r, c, l),
                                  "seconds": round(t, 2)}}


# ----------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    """The oracle as the reference arm: every step runs the same algorithm
    as our arm (Winograd, cutoff and precision of the workload) on one of the
    49 level-2 sub-products of the n^3 product (winograd_subproduct); the
    whole-product rate is 2 n^3 / (49 t).  Rank 0 only."""
    if rank != 0:
        return
    from paper_1410_1599_gb300 import inputs as gen

    n, p = a.n, a.prec
    A = gen.uniform_pm1(n, n, p, 3, -16, 16)
    B = gen.uniform_pm1(n, n, p, 4, -16, 16)
    from oracle import oracle as orc
    threads = orc.max_threads()
    for s in range(a.warmup):
        winograd_subproduct(A, B, a.cutoff)
    ts = []
    for s in range(a.steps):
        t, h, _ = winograd_subproduct(A, B, a.cutoff)
        ts.append(t)
    t = sum(ts) / len(ts)
    value = 2.0 * n ** 3 / (49 * t) / 1e9
    line = {"impl": "reference", "metric": "eff. MP GFLOP/s (2mln/t)", "value": round(value, 6),
            "unit": "GFLOP/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": round(t * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mp%d" % p, "data": "synthetic",
            "config": workload_config(a),
            "cpu_baseline": {"value": round(value, 6), "unit": "GFLOP/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "per step: Winograd (cutoff %d) on one of the 49 level-2 "
                                       "sub-products (a %d^3 product); whole-product rate = 2 n^3 / (49 t)"
                                       % (a.cutoff, h)},
            "e2e": {"value": round(value, 6), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    rank, world, local = dist_env()
    if a.split:
        import torch
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        n_s, p_s = (a.n if a.n != 2048 else 4096), (a.prec if a.prec != 512 else 1024)
        print(json.dumps({"split_form": split_run(n_s, p_s),
                          "split_form_u11": split_run(n_s, p_s, with_simple=False, exp_lo=0, exp_hi=0,
                                                      with_exact=False)}), flush=True)
        return
    if a.cond:
        import torch
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps({"cond1_lotkin": cond_run(a.lu_n)}), flush=True)
        return
    if a.lotkin:
        import torch
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps({"lotkin": lotkin_run(a.lu_n)}), flush=True)
        return
    if a.lu_sweep:
        import torch
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps({"lu_sweep": lu_sweep_run(a.lu_n)}), flush=True)
        return
    if a.paper:
        import torch
        from paper_1410_1599_gb300 import binding as mp
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        stream = torch.cuda.Stream()
        mp.set_stream(stream)
        print(json.dumps({"paper_section4": paper_run(stream)}), flush=True)
        return
    if a.serve:
        import torch
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        print(json.dumps({"serving": serve_run(a.serve_requests),
                          "serving_repeated_shapes": serve_repeat_run()}), flush=True)
        return
    if a.configs:
        import torch
        from paper_1410_1599_gb300 import binding as mp
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        stream = torch.cuda.Stream()
        mp.set_stream(stream)
        print(json.dumps({"configs": configs_run(stream)}), flush=True)
        return
    if a.lu:
        import torch
        from paper_1410_1599_gb300 import binding as mp
        from paper_1410_1599_gb300 import build as libbuild
        libbuild.build()
        torch.cuda.set_device(local)
        runs = [lu_run(a.lu_n, p, mp.WINOGRAD, kind=kind) for kind in ("well", "lotkin") for p in (256, 1024)]
        print(json.dumps({"lu": runs}), flush=True)
        return
    if a.impl == "reference":
        run_reference(a, rank, world)
    else:
        run_ours(a, rank, world, local)


if __name__ == "__main__":
    main()
