"""Benchmark: filtered nnz*R*p updates/s of the accelerated-spectral-clustering
hot path on one GB300 (or N GPUs, one process each).

One step = one pass of the whole path over one batch of synthetic input
(a seeded stochastic-block-model graph and a block of random signals already
resident in device memory):
  CSR build from the edge list -> lambda_N by Lanczos (40 steps) ->
  moment sweep (p orders, on the count's own probe block) -> dichotomy for
  lambda_k -> coefficients -> filter sweep (p orders, on R) ->
  row-normalised features; both sweeps store their blocks as the workload
  says (BF16 at the default) and accumulate in FP32.
Updates counted per step: (nnz_off + N) * R * p for each of the two sweeps.

Besides the contract's keys the JSON line carries: the roofline of the
dominant sweep kernel (and of each variant) with its ncu DRAM traffic, the
measured ceiling of its random-row gathers, where a step's device time goes,
the same step with FP32 blocks, the end-to-end timing from pinned host
buffers, k-means on the step's features (tensor cores with split and with
single TF32 products, CUDA cores), the method end to end against the
generating communities (and on the normalised Laplacian and the stability
measure up to 200k nodes), the CPU oracle's rate, the filter's error against
the FP64 oracle, and the SM clocks sampled during the timed region.

Default workload ("sbm1m"): N = 1,000,000, k = 100 equal communities, mean
degree 30, c_out/c_in = 0.08, unit weights, R = 128 signals, p = 200, filter
blocks stored in BF16 with FP32 accumulation; the same step with FP32 blocks
is timed beside it. Inputs (graph 0.25 GB CSR, blocks 0.5 GB) are larger
than L2, so no flush is needed between steps.

--impl reference times the CPU FP64 oracle (the correctness reference; there
is no other implementation) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (N, k, mean degree, eps, R, p, storage)
    "sbm1m": dict(n=1_000_000, k=100, deg=30.0, eps=0.08, R=128, p=200, storage="bf16", graph_seed=1003,
                  r_seed=2003),
    "sbm100k": dict(n=100_000, k=20, deg=20.0, eps=0.1, R=64, p=100, storage="f32", graph_seed=1002, r_seed=2002,
                    sizes=(2000, 8000)),
    "sbm1k": dict(n=1000, k=10, deg=16.0, eps=0.05, R=14, p=50, storage="f32", graph_seed=1001, r_seed=2001),
    # differentiable filter: 10-NN Gaussian-kernel graph of a 10-component mixture in d = 8
    "knn200k": dict(n=200_000, k=10, dim=8, knn=10, sigma=1.0, R=64, p=80, storage="f32", graph_seed=1004,
                    r_seed=2004, g_seed=3000),
    # many graphs: 256 SBMs of uneven size, one per-graph cutoff each
    "batch256": dict(n_graphs=256, R=32, p=120, storage="bf16", graph_seed=10000, r_seed=2005),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sbm1m", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-kmeans", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other workloads' legs (sbm1k, sbm100k, knn200k, batch256) of the default run")
    ap.add_argument("--kernel-case", default=None,
                    help="profiling aid: MODE:STORAGE:SLAB:WARPS:CARVEOUT[:KERNEL] (MODE moments|clenshaw|forward|adjoint|"
                         "kmeans|batched, STORAGE f32|bf16, KERNEL tiled|direct|persistent) runs two sweeps of --case-orders orders over one column slab of "
                         "the workload and exits")
    ap.add_argument("--case-orders", type=int, default=6)
    ap.add_argument("--case-graphs", type=int, default=0,
                    help="kernel case 'batched': only the first K graphs of the batch (0: all), for small captures")
    ap.add_argument("--filter-algo", default="auto", choices=["auto", "clenshaw", "forward"],
                    help="algorithm of the filter sweep (auto: Clenshaw for FP32 blocks, forward otherwise); "
                         "the moment sweep is always the forward recurrence")
    ap.add_argument("--compare-storage", action="store_true",
                    help="also time the step with FP16 blocks in the filter")
    return ap.parse_args()


def run_kernel_case(args, wl):
    """Two sweeps of one kernel variant over one slab of the workload, for ncu."""
    import torch

    import paper_1509_08863_gb300 as sf
    from paper_1509_08863_gb300 import build as sfbuild

    sfbuild.build()
    fields = args.kernel_case.split(":")
    mode, stor, slab, warps, carve = fields[:5]
    kind = {"tiled": sf.SWEEP_TILED, "direct": sf.SWEEP_DIRECT,
            "persistent": sf.SWEEP_PERSISTENT}[fields[5] if len(fields) > 5 else "tiled"]
    slab, warps, carve = int(slab), int(warps), int(carve)
    st = sf.BF16 if stor == "bf16" else sf.F32
    dev = torch.device("cuda")
    p = args.case_orders
    if mode == "kmeans":
        # Lloyd assignments on N unit rows of R columns (the workload's feature shape), k centroids
        gen = torch.Generator(device="cuda").manual_seed(0)
        F = torch.randn(wl["n"], wl["R"], device=dev, generator=gen)
        F /= F.norm(dim=1, keepdim=True)
        for _ in range(2):
            sf.kmeans(F, F[:wl["k"]].clone(), 2, sf.KMEANS_TENSOR)
        torch.cuda.synchronize()
        print(json.dumps({"kernel_case": args.kernel_case, "status": "ok"}))
        return 0
    if mode == "adjoint":
        # one slab of the filter's reverse mode on the kNN graph (p = case_orders)
        from paper_1509_08863_gb300 import synth

        src, dst, w, _, _ = synth.knn_mixture_edges(wl["n"], wl["k"], wl["dim"], wl["knn"], wl["sigma"], 3.0,
                                                    wl["graph_seed"])
        g = sf.csr_build(wl["n"], torch.as_tensor(src, device=dev), torch.as_tensor(dst, device=dev),
                         torch.as_tensor(w, device=dev))
        _, lh = sf.lambda_max_estimate(g, 60, None, seed=11)
        Rs = torch.as_tensor(synth.gaussian_block(wl["n"], slab, wl["r_seed"]), dtype=torch.float32, device=dev)
        Gs = torch.as_tensor(synth.standard_normal_block(wl["n"], slab, wl["g_seed"]), dtype=torch.float32,
                             device=dev)
        a = sf.cheb_coeffs(lh, 0.02 * lh, p, True)[0]
        o = sf.Opts(slab_cols=slab, block_warps=warps, carveout_pct=carve, sweep_kernel=kind)
        for _ in range(2):
            sf.cheb_filter_backward(g, lh, a, Rs, Gs, False, o)
        torch.cuda.synchronize()
        sf.device_check()
        print(json.dumps({"kernel_case": args.kernel_case, "orders": p, "status": "ok"}))
        return 0
    if mode == "batched":
        # the 256-graph batch, one forward sweep launch per order for all graphs (p = case_orders)
        from paper_1509_08863_gb300 import synth

        graphs, _ = synth.batched_sbm(wl["n_graphs"], wl["graph_seed"])
        if args.case_graphs > 0:
            graphs = graphs[:args.case_graphs]
        gs = [sf.csr_build(gr.n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
              for gr in graphs]
        lams = np.array([sf.lambda_max_estimate(g, 40, None, seed=11)[1] for g in gs])
        b = sf.batch_build(gs)
        n_tot = b.info()[0]
        Rb = torch.as_tensor(synth.gaussian_block(n_tot, slab, wl["r_seed"]), dtype=torch.float32, device=dev)
        coeffs = np.stack([sf.cheb_coeffs(lams[i], 0.1 * lams[i], p, True)[0] for i in range(len(gs))])
        o = sf.Opts(storage=st, slab_cols=slab, block_warps=warps, carveout_pct=carve, sweep_kernel=kind)
        for _ in range(2):
            sf.cheb_filter_batched(b, lams, coeffs, Rb, o)
        torch.cuda.synchronize()
        sf.device_check()
        print(json.dumps({"kernel_case": args.kernel_case, "orders": p, "status": "ok"}))
        return 0
    algo = {"moments": sf.ALGO_CLENSHAW, "clenshaw": sf.ALGO_CLENSHAW, "forward": sf.ALGO_FORWARD}[mode]
    gr, R = make_inputs(wl)
    g = sf.csr_build(wl["n"], torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    Rs = torch.as_tensor(R[:, :slab], dtype=torch.float32, device=dev).contiguous()
    _, lh = sf.lambda_max_estimate(g, 40, None, seed=11)
    a = sf.cheb_coeffs(lh, 0.05 * lh, p, True)
    o = sf.Opts(storage=st, algo=algo, slab_cols=slab, block_warps=warps, carveout_pct=carve, sweep_kernel=kind)
    for _ in range(2):
        if mode == "moments":
            sf.cheb_moments(g, lh, Rs, p, o)
        else:
            sf.cheb_filter(g, lh, a, Rs, o)
    torch.cuda.synchronize()
    sf.device_check()
    print(json.dumps({"kernel_case": args.kernel_case, "orders": p, "status": "ok"}))
    return 0


def make_inputs(wl, rank=0):
    from paper_1509_08863_gb300 import synth

    if "sizes" in wl:
        sizes = synth.community_sizes_uniform(wl["n"], wl["k"], wl["sizes"][0], wl["sizes"][1], wl["graph_seed"])
    else:
        sizes = synth.community_sizes_equal(wl["n"], wl["k"])
    gr = synth.sbm_edges(wl["n"], sizes, wl["deg"], wl["eps"], seed=wl["graph_seed"])
    R = synth.standard_normal_block(wl["n"], wl["R"], seed=wl["r_seed"] + 7919 * rank)
    R /= np.sqrt(wl["R"])
    return gr, R


def make_count_signals(wl, rank=0):
    """The eigenvalue count's own probe block (§4.1 draws the filtered signals
    R in step 4, after lambda_k is estimated in step 2): same law, other seed."""
    from paper_1509_08863_gb300 import synth

    Rc = synth.standard_normal_block(wl["n"], wl["R"], seed=wl["r_seed"] + 1 + 7919 * rank)
    Rc /= np.sqrt(wl["R"])
    return Rc


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


SWEEP_SOURCES = ("sf_internal.cuh", "sf_step.cuh", "sf_cheb.cu", "sf_sell.cu", "sf_adjoint.cu")


def kernel_source_hash(sources=SWEEP_SOURCES):
    """Hash of the CUDA sources a committed ncu figure depends on: the figure is
    used only while the hash matches the one recorded with it."""
    h = hashlib.sha256()
    for fn in sources:
        with open(os.path.join(ROOT, "paper_1509_08863_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profile(workload, variant):
    """DRAM bytes per sweep launch of a kernel variant from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"cheb_step_{workload}_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_sha") == kernel_source_hash(tuple(d.get("sources", SWEEP_SOURCES))):
            return d["variants"][variant]["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


# ----------------------------------------------------------------- reference arm
def run_reference(args, wl):
    import oracle

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    gr, R = make_inputs(wl)
    g = oracle.csr_build(wl["n"], gr.src, gr.dst, gr.w)
    lam = 2.0 * float(oracle.strength(g).max())
    try:  # the OpenMP build on every host core (identical results to the plain build)
        oracle.build_parallel()
        par = True
        threads = oracle.threads(parallel=True)
    except Exception:
        par = False
        threads = 1
    # a bounded sample per step: every order on a few columns (all cores), or a few orders on one thread
    p_ref = wl["p"] if par else (4 if wl["n"] >= 500_000 else max(1, min(wl["p"], 20)))
    a = oracle.cheb_coeffs(lam, 0.1 * lam, p_ref, True)
    cols = min(8, wl["R"])  # as the cpu_baseline leg of our own arm
    blk = np.ascontiguousarray(R[:, :cols])
    units = (g.nnz + wl["n"]) * cols * p_ref
    for _ in range(args.warmup):
        oracle.cheb_filter(g, lam, a, blk, parallel=par)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.cheb_filter(g, lam, a, blk, parallel=par)
        ts.append(time.perf_counter() - t0)
    t = sum(ts) / len(ts)
    v = units / t
    sample = (f"{cols} of {wl['R']} signal columns, all {wl['n']} nodes, {p_ref} Chebyshev orders per step "
              f"(oracle_cheb_filter, FP64, {'OpenMP build' if par else 'plain build'}, {threads} threads)")
    out = {
        "impl": "reference",
        "metric": "filtered nnz*R*p updates/s",
        "value": v,
        "unit": "updates/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": wl["n"], "R": wl["R"], "p": wl["p"], "k": wl["k"],
                   "mean_degree": wl["deg"], "c_out_over_c_in": wl["eps"]},
        "cpu_baseline": {"value": v, "unit": "updates/s", "cores": threads, "host_cores": host_cores(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ----------------------------------------------------------------- our arm
def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    if args.kernel_case:
        return run_kernel_case(args, wl)
    if args.workload == "knn200k":
        print(json.dumps(run_knn_grad(args, wl)))
        return 0
    if args.workload == "batch256":
        print(json.dumps(run_batch(args, wl)))
        return 0

    import torch

    import paper_1509_08863_gb300 as sf
    from paper_1509_08863_gb300 import build as sfbuild
    from paper_1509_08863_gb300 import sharded

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if "WORLD_SIZE" in os.environ:  # launched by torch.distributed.run (any world size)
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist = None
    if rank == 0:
        sfbuild.build()
    if dist:
        dist.barrier()
    dev = torch.device("cuda", local)
    gr, R = make_inputs(wl, rank)
    n, eta, p, k = wl["n"], wl["R"], wl["p"], wl["k"]
    storage = sf.BF16 if wl["storage"] == "bf16" else sf.F32
    src_h = torch.from_numpy(gr.src).pin_memory()
    dst_h = torch.from_numpy(gr.dst).pin_memory()
    R_h = torch.from_numpy(R.astype(np.float32)).pin_memory()
    Rc_h = torch.from_numpy(make_count_signals(wl, rank).astype(np.float32)).pin_memory()
    src_d, dst_d, R_d, Rc_d = src_h.to(dev), dst_h.to(dev), R_h.to(dev), Rc_h.to(dev)
    stream = torch.cuda.current_stream()

    # tile shapes from the autotuner (untimed; cached per graph size)
    g0 = sf.csr_build(n, src_d, dst_d, None)
    tuned = {storage: sf.autotune(g0, eta, storage, 1)}
    g0.free()

    filter_algo = {"auto": sf.ALGO_AUTO, "forward": sf.ALGO_FORWARD, "clenshaw": sf.ALGO_CLENSHAW}[args.filter_algo]

    def opts_for(st, algo=sf.ALGO_CLENSHAW):
        t = tuned[st]
        return sf.Opts(storage=st, algo=algo, slab_cols=t.slab_cols, block_warps=t.block_warps,
                       blocks_per_sm=t.blocks_per_sm, carveout_pct=t.carveout_pct, l2_window=t.l2_window,
                       sweep_kernel=t.sweep_kernel)

    def step(src, dst, Rc, Rt, st, collect=None, marks=None, before_filter=None):
        """One pass of the path: the count's moments on the probe block Rc, the
        filter on R. `st` is the block storage of both sweeps (FP16 applies to
        the filter, whose moments then use BF16 blocks). `marks`, when given,
        collects (stage, CUDA event) pairs after each stage. `before_filter` is
        called once the step has made its last host round trip (after the
        coefficients), just before the filter sweep is enqueued."""
        def mark(name):
            if marks is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                marks.append((name, e))

        mark("start")
        g = sf.csr_build(n, src, dst, None)
        mark("csr_build")
        _, lh = sf.lambda_max_estimate(g, 40, None, seed=11)
        mark("lambda_max_estimate")
        mst = sf.BF16 if st == sf.F16 else st
        if mst not in tuned:
            tuned[mst] = sf.autotune(g, eta, mst, 1)
        mu = sf.cheb_moments(g, lh, Rc, p, opts_for(mst))
        if dist:  # columns are sharded over ranks: moments add up
            mu = sharded.combine_moments(mu, device=dev)
        mark("cheb_moments")
        lk = sf.dichotomy(mu, p, lh, k - 0.5, True, 40, 1e-9)
        a = sf.cheb_coeffs(lh, lk, p, True)
        mark("dichotomy_and_coeffs")
        if st not in tuned:
            tuned[st] = sf.autotune(g, eta, st, 1)
        if before_filter is not None:
            before_filter()
        Y = sf.cheb_filter(g, lh, a, Rt, opts_for(st, filter_algo))[0]
        mark("cheb_filter")
        if dist:  # row norms run over every rank's columns
            F = sharded.normalize_rows_sharded(Y, sf.row_sumsq, lambda y, tot: sf.features_scaled(y, tot, out=y))
        else:
            F = sf.features(Y, True, out=Y)
        mark("features")
        if collect is not None:
            collect.update(lam_hat=lh, lam_k=lk, nnz=g.nnz, Y=Y)
        g.free()
        return F

    info = {}
    F = step(src_d, dst_d, Rc_d, R_d, storage, info)
    torch.cuda.synchronize()
    nnz = info["nnz"]
    updates = 2.0 * (nnz + n) * eta * p

    # inputs smaller than L2: overwrite a buffer larger than L2 between timed steps
    in_bytes = 4 * (src_h.numel() + dst_h.numel() + R_h.numel() + Rc_h.numel())
    flush = torch.zeros(64 << 20, dtype=torch.float32, device=dev) if in_bytes < (256 << 20) else None

    def timed(st, steps, warmup):
        """Mean device time of `steps` steps on device-resident inputs (CUDA
        events around each step, on the launching stream)."""
        for _ in range(warmup):
            step(src_d, dst_d, Rc_d, R_d, st)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        l0 = sf.launch_count()
        torch.cuda.nvtx.range_push("timed")
        for i in range(steps):
            ev[i][0].record(stream)
            step(src_d, dst_d, Rc_d, R_d, st)
            ev[i][1].record(stream)
            if flush is not None:  # between steps, outside the timed spans
                flush.add_(1)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        launches = sf.launch_count() - l0
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, launches

    def timed_e2e(st, steps, warmup):
        """Steps fed from pinned host buffers, features read back to pinned host
        memory, all inside the timed region. The copies run on a second stream
        and are enqueued while a step's filter sweep runs (after its last host
        round trip, so that the step's own small reads never queue behind them):
        the previous step's features go back to the host and the next step's
        inputs come in (two device input buffers). Only the first step's inputs
        and the last step's features are not overlapped."""
        cs = torch.cuda.Stream(device=dev)
        host = (src_h, dst_h, Rc_h, R_h)
        bufs = [tuple(torch.empty(h.shape, dtype=h.dtype, device=dev) for h in host) for _ in range(2)]
        host_out = [torch.empty((n, eta), dtype=torch.float32).pin_memory() for _ in range(2)]

        def run(total):
            start = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            ev_in = [torch.cuda.Event(), torch.cuda.Event()]
            ev_done = [None, None]
            prev = [None, None, 0]  # output, its event, its step index
            cs.wait_event(start)
            with torch.cuda.stream(cs):
                for d_, h_ in zip(bufs[0], host):
                    d_.copy_(h_, non_blocking=True)
                ev_in[0].record(cs)

            def read_back(out, ev, i):
                cs.wait_event(ev)
                out.record_stream(cs)
                host_out[i % 2].copy_(out, non_blocking=True)

            for i in range(total):
                b = i % 2

                def overlap():
                    with torch.cuda.stream(cs):
                        if prev[0] is not None:
                            read_back(*prev)
                        if i + 1 < total:  # buffer (i + 1) % 2 was last read by step i - 1
                            nb = (i + 1) % 2
                            if ev_done[nb] is not None:
                                cs.wait_event(ev_done[nb])
                            for d_, h_ in zip(bufs[nb], host):
                                d_.copy_(h_, non_blocking=True)
                            ev_in[nb].record(cs)

                stream.wait_event(ev_in[b])
                out = step(*bufs[b], st, before_filter=overlap)
                done = torch.cuda.Event()
                done.record(stream)
                ev_done[b] = done
                prev[:] = [out, done, i]
            with torch.cuda.stream(cs):
                read_back(*prev)
            fin = torch.cuda.Event()
            fin.record(cs)
            stream.wait_event(fin)
            end = torch.cuda.Event(enable_timing=True)
            end.record(stream)
            return start, end

        run(max(warmup, 1))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        s0, s1 = run(steps)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1) / steps
        if dist:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    # main timed region (device-resident inputs) with kernel timing and clocks
    clk = ClockSampler(local if world == 1 else int(os.environ.get("LOCAL_RANK", "0")))
    for _ in range(args.warmup):
        step(src_d, dst_d, Rc_d, R_d, storage)
    torch.cuda.synchronize()
    clk.start()
    sf.profile_begin()
    ms, launches = timed(storage, args.steps, 0)
    k_launches, k_ms, k_bytes = sf.profile_end()
    variants = sf.profile_variants()
    clocks = clk.stop()
    sf.device_check()
    value = updates * world / (ms * 1e-3)

    # where one step's device time goes (one extra, untimed step with events between stages)
    marks = []
    step(src_d, dst_d, Rc_d, R_d, storage, marks=marks)
    torch.cuda.synchronize()
    stages = {name: marks[i - 1][1].elapsed_time(e) for i, (name, e) in enumerate(marks) if i > 0}

    # the same run with FP32 blocks in both sweeps
    fp32 = None
    if storage != sf.F32 and not args.no_fp32:
        ms32, _ = timed(sf.F32, max(3, args.steps // 2), 1)
        fp32 = {"value": updates * world / (ms32 * 1e-3), "ms_per_step": ms32,
                "speedup_of_storage": ms32 / ms}
    f16 = None
    if args.compare_storage and storage != sf.F16:
        ms16, _ = timed(sf.F16, max(3, args.steps // 2), 1)
        f16 = {"value": updates * world / (ms16 * 1e-3), "ms_per_step": ms16,
               "note": "FP16 blocks in the filter, BF16 blocks in the moment sweep"}
    # end to end from pinned host buffers, features copied back
    e2e = None
    if not args.no_e2e:
        mse = timed_e2e(storage, max(3, args.steps // 2), 1)
        e2e = {"value": updates * world / (mse * 1e-3), "unit": "updates/s", "ms_per_step": mse,
               "copies": "on a second stream, enqueued during each step's filter sweep: the previous step's features "
                         "out, the next step's inputs in (two input buffers)",
               "h2d_bytes_per_step": int(src_h.numel() * 4 + dst_h.numel() * 4 + R_h.numel() * 4 +
                                         Rc_h.numel() * 4),
               "d2h_bytes_per_step": int(n * eta * 4)}

    # k-means on the step's features (§4.1 step 6; measured apart from the step)
    kmeans = None
    if not args.no_kmeans and world == 1:
        kmeans = run_kmeans_leg(sf, info["Y"], k, wl["r_seed"] + 5, 20)

    # the method end to end on this graph (§4.1: count, filter, features, k-means; FP32 blocks) against the
    # generating communities; where the graph is small enough also on the normalised Laplacian (footnote of
    # §2.1) and the stability measure of §4.3
    clustering = clustering_norm = stability = None
    if not args.no_kmeans and world == 1:
        gq = sf.csr_build(n, src_d, dst_d, None)
        _, lq = sf.lambda_max_estimate(gq, 40, None, seed=11)
        clustering = cluster_recovery(sf, gq, lq, R_d, k, p, gr.labels, seed=wl["r_seed"])
        if n <= 200_000:
            stability = stability_leg(sf, gq, lq, p, n, eta, k, seed=wl["r_seed"])
            gn = gq.normalized()
            _, ln = sf.lambda_max_estimate(gn, 40, None, seed=11)
            clustering_norm = cluster_recovery(sf, gn, ln, R_d, k, p, gr.labels, seed=wl["r_seed"])
            gn.free()
        gq.free()

    # accuracy of this step's features/filter against the FP64 oracle on one column
    hbm, peak_kind = peaks()

    def roof_of(name, n_l, ms_, by_):
        gbs = by_ / (ms_ * 1e-3) / 1e9 if ms_ > 0 else 0.0
        return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                "traffic": traffic_from_profile(args.workload, name),
                "kernel": (f"sddmm_kernel ({name})" if name.startswith("adjoint") else f"cheb_step_kernel ({name})"),
                "launches_timed": n_l, "avg_launch_ms": ms_ / max(n_l, 1), "bytes_per_launch": by_ / max(n_l, 1),
                "share_of_sweep_time": ms_ / k_ms if k_ms > 0 else None, "peak_source": f"{peak_kind} hbm_gbs"}

    by_variant = {name: roof_of(name, *v) for name, v in variants.items()}
    dominant = max(variants.items(), key=lambda kv: kv[1][1])[0] if variants else None
    roof = by_variant.get(dominant) if dominant else None

    # the gather pattern's own ceiling: random rows of the slab width from a block
    # of N rows, timed alone (untimed by the step clock)
    gather = None
    st_b = 2 if storage != sf.F32 else 4
    t_main = tuned.get(storage)
    if t_main is not None and t_main.slab_cols * st_b in (32, 64, 128, 256):
        rb = t_main.slab_cols * st_b
        deg = max(4, int(round(nnz / n / 4.0)) * 4)
        rps = sf.gather_ceiling(n, rb, deg, 10)
        at_ceiling = nnz / rps * 1e3
        gather = {"rows_per_s": rps, "row_bytes": rb, "table_rows": n, "deg": deg,
                  "launch_ms_at_ceiling": at_ceiling,
                  "frac_of_ceiling": {name: at_ceiling / v["avg_launch_ms"] for name, v in by_variant.items()},
                  "note": "sf_gather_ceiling: the sweep's random-row gathers with each row's sums written back "
                          "(nnz_off rows per launch)"}
        # the gathers with nothing else in flight (one float written per row): the bound any kernel that
        # gathers these rows meets, and the HBM fraction of the algorithmic bytes it allows
        rps0 = sf.gather_rate(n, rb, deg, 10, write_rows=False)
        at0 = nnz / rps0 * 1e3
        gather["gathers_alone"] = {
            "rows_per_s": rps0, "launch_ms": at0,
            "frac_of_rate": {name: at0 / v["avg_launch_ms"] for name, v in by_variant.items()},
            "roofline_frac_bound": {name: v["bytes_per_launch"] / (at0 * 1e-3) / 1e9 / v["peak"]
                                    for name, v in by_variant.items() if v.get("bytes_per_launch")},
            "note": "sf_gather_rate(write_rows=0)"}

    result = {
        "metric": "filtered nnz*R*p updates/s",
        "value": value,
        "unit": "updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"{wl['storage']}-storage/f32-compute",
        "data": "synthetic",
        "config": {"workload": args.workload, "N": n, "nnz_off": nnz, "R": eta, "p": p, "k": k,
                   "mean_degree": wl["deg"], "c_out_over_c_in": wl["eps"],
                   "block_storage": wl["storage"], "accumulation": "f32", "filter_algo": args.filter_algo,
                   "updates_counted": "(nnz_off + N) * R * p for each of the step's two sweeps: the count's "
                                      "moment sweep on its probe block and the filter sweep on R",
                   "tiles": {("f32", "bf16", "f16")[k]: {"slab_cols": v.slab_cols, "block_warps": v.block_warps,
                                                                  "carveout_pct": v.carveout_pct, "l2_window": v.l2_window,
                                                                  "sweep_kernel": ("auto", "tiled", "direct")[v.sweep_kernel]}
                             for k, v in tuned.items()},
                   "sweeps_per_step": 2,
                   "l2": ("inputs larger than L2 (no flush)" if flush is None else
                          "inputs smaller than L2: a 256 MB buffer is overwritten between timed steps"),
                   "signals": "the count's probe block and the filtered block R are drawn independently (N(0, 1/R) each)",
                   "parallelism": (f"column shards x{world}: each rank filters its own {wl['R']} signals of one "
                                   f"{wl['R'] * world}-signal block; moments and row norms all-reduced")
                   if world > 1 else "single GPU"},
        "gpu_launches": launches,
        "roofline": roof,
        "gather_ceiling": gather,
        "stages_ms": stages,
        "kmeans": kmeans,
        "clustering": clustering,
        "clustering_normalized_laplacian": clustering_norm,
        "stability": stability,
        "roofline_by_variant": by_variant,
        "clocks": clocks,
        "e2e": e2e,
        "fp32_storage": fp32,
        "fp16_storage": f16,
        "lam_hat": info["lam_hat"],
        "lam_k_estimate": info["lam_k"],
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"], result["accuracy"] = cpu_baseline_and_accuracy(gr, R, info, wl, sf, dev)
    if rank == 0 and world == 1 and not args.no_configs and args.workload == "sbm1m":
        result["configs"] = other_configs(args, sf)
    if rank == 0:
        print(json.dumps(result))
    if dist:
        dist.destroy_process_group()
    return 0


def tf32_peak():
    """Dense TF32 tensor peak: the measured BF16 burst peak times the nominal
    TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16_tflops x 1.1/2.25"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback 1.9 PFLOP/s bf16 x 1.1/2.25"


def run_kmeans_leg(sf, Fk, k, seed, max_iter):
    """Lloyd's k-means on feature rows Fk (N x d, FP32, on the device) from k
    seeded random rows: tensor cores (when the shape allows) vs CUDA cores,
    the same labels; the distance kernel's roofline."""
    import torch

    n, d = Fk.shape
    rng = np.random.default_rng(seed)
    C0 = Fk[torch.as_tensor(rng.choice(n, k, replace=False), device=Fk.device)].contiguous().clone()
    tc_ok = d % 32 == 0 and 32 <= d <= 128 and k <= 128
    out = {"rows": n, "d": d, "k": k, "max_iter": max_iter, "init": "k seeded random rows"}
    res = {}
    for name, mode in (("tensor_cores", sf.KMEANS_TENSOR if tc_ok else None),
                       ("tensor_cores_single_product", sf.KMEANS_TENSOR_SINGLE if tc_ok else None),
                       ("cuda_cores", sf.KMEANS_CUDA_CORES)):
        if mode is None:
            continue
        sf.kmeans(Fk, C0, 2, mode)  # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sf.profile_begin()
        e0.record()
        lab, C, it, inertia = sf.kmeans(Fk, C0, max_iter, mode)
        e1.record()
        torch.cuda.synchronize()
        sf.profile_end()
        v = sf.profile_variants()
        ms = e0.elapsed_time(e1)
        res[name] = lab
        ent = {"ms": ms, "assignments": it, "ms_per_assignment": ms / it, "inertia": inertia}
        if "kmeans_tc_f32" in v:
            nl, kms, by = v["kmeans_tc_f32"]
            t = kms / nl * 1e-3
            mma = 3 if mode == sf.KMEANS_TENSOR else 1  # split operands: hi.hi + hi.lo + lo.hi
            hbm, kind = peaks()
            tfp, tkind = tf32_peak()
            ent["distance_kernel"] = {
                "avg_launch_ms": kms / nl, "launches": nl,
                "hbm": {"achieved": by / nl / t / 1e9, "peak": hbm, "unit": "GB/s", "frac": by / nl / t / 1e9 / hbm,
                        "peak_source": f"{kind} hbm_gbs"},
                "tensor": {"achieved": mma * 2.0 * n * k * d / t / 1e12, "peak": tfp, "unit": "TFLOP/s",
                           "frac": mma * 2.0 * n * k * d / t / 1e12 / tfp, "peak_source": tkind,
                           "products_per_pair": mma},
                "bound": "hbm"}
        out[name] = ent
    if len(res) > 1:
        out["labels_equal"] = all(bool(torch.equal(lab, res["cuda_cores"])) for lab in res.values())
    return out


def _clock_timed(fn, steps, warmup, sf, flush_l2=False):
    """Mean device time of fn over `steps` calls (CUDA events around each call);
    with flush_l2, a 256 MB buffer is overwritten between calls, outside the
    timed spans (for inputs smaller than L2)."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda") if flush_l2 else None
    clk = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clk.start()
    sf.profile_begin()
    l0 = sf.launch_count()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.nvtx.range_push("timed")
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
        if flush is not None:
            flush.add_(1)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    launches = sf.launch_count() - l0
    sf.profile_end()
    variants = sf.profile_variants()
    clocks = clk.stop()
    sf.device_check()
    return sum(a.elapsed_time(b) for a, b in ev) / steps, launches, variants, clocks


def _roof_variants(variants, workload):
    hbm, kind = peaks()
    out = {}
    tot = sum(v[1] for v in variants.values()) or 1.0
    for name, (n_l, ms, by) in variants.items():
        gbs = by / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        out[name] = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "traffic": traffic_from_profile(workload, name), "kernel": (f"sddmm_kernel ({name})" if name.startswith("adjoint") else f"cheb_step_kernel ({name})"),
                     "launches_timed": n_l, "avg_launch_ms": ms / max(n_l, 1), "share_of_sweep_time": ms / tot,
                     "peak_source": f"{kind} hbm_gbs"}
    dom = max(out.items(), key=lambda kv: kv[1]["share_of_sweep_time"])[0] if out else None
    return (out[dom] if dom else None), out


def run_knn_grad(args, wl):
    """Forward filter + reverse mode (edge weights, coefficients) on the 10-NN
    Gaussian-kernel graph; updates = 3 sweeps x (nnz + N) x R x p per step
    (the filter, its recomputation inside the backward call, the adjoint)."""
    import torch

    import paper_1509_08863_gb300 as sf
    from paper_1509_08863_gb300 import build as sfbuild
    from paper_1509_08863_gb300 import synth

    sfbuild.build()
    dev = torch.device("cuda")
    n, eta, p = wl["n"], wl["R"], wl["p"]
    src, dst, w, labels, _ = synth.knn_mixture_edges(n, wl["k"], wl["dim"], wl["knn"], wl["sigma"], 3.0,
                                                     wl["graph_seed"])
    g = sf.csr_build(n, torch.as_tensor(src, device=dev), torch.as_tensor(dst, device=dev),
                     torch.as_tensor(w, device=dev))
    nnz = g.nnz
    _, lh = sf.lambda_max_estimate(g, 60, None, seed=11)
    R = torch.as_tensor(synth.gaussian_block(n, eta, wl["r_seed"]), dtype=torch.float32, device=dev)
    G = torch.as_tensor(synth.standard_normal_block(n, eta, wl["g_seed"]), dtype=torch.float32, device=dev)
    mu = sf.cheb_moments(g, lh, R, p)
    lk = sf.dichotomy(mu, p, lh, wl["k"] - 0.5)
    a = sf.cheb_coeffs(lh, lk, p, True)[0]
    opts = sf.Opts()

    def step():
        sf.cheb_filter(g, lh, a[None, :], R, opts)
        sf.cheb_filter_backward(g, lh, a, R, G, False, opts)

    ms, launches, variants, clocks = _clock_timed(step, args.steps, args.warmup, sf, flush_l2=True)
    updates = 3.0 * (nnz + n) * eta * p
    roof, by_variant = _roof_variants(variants, args.workload)
    # directional finite difference at full size: l(W + h D) - l(W - h D) vs <grad, D>
    gv, ga, _ = sf.cheb_filter_backward(g, lh, a, R, G, False, opts)
    val0 = g.csr()[2]
    rp, ci = g.csr()[0].cpu().numpy(), g.csr()[1].cpu().numpy()
    rows = np.repeat(np.arange(n), np.diff(rp))
    rng = np.random.default_rng(7)
    # relative perturbation of each undirected edge weight (weights span many decades)
    und = rng.standard_normal(len(ci)) * val0.cpu().numpy()
    # symmetric direction: entries (u, v) and (v, u) move together
    key_lo, key_hi = np.minimum(rows, ci), np.maximum(rows, ci)
    order = np.lexsort((key_hi, key_lo))
    d = np.empty(len(ci))
    d[order] = np.repeat(und[order][::2], 2)
    D = torch.as_tensor(d, dtype=torch.float32, device=dev)
    h = 1e-3

    def loss(vals):
        g.set_values(vals.contiguous())
        Y = sf.cheb_filter(g, lh, a[None, :], R, sf.Opts(algo=sf.ALGO_FORWARD))[0]
        return float((Y.double() * G.double()).sum())

    lp, lm = loss(val0 + h * D), loss(val0 - h * D)
    g.set_values(val0.contiguous())
    fd = (lp - lm) / (2 * h)
    an = float((gv.double() * D.double()).sum()) / 2.0  # each undirected edge appears twice in D and gv
    out = {
        "metric": "filtered nnz*R*p updates/s", "value": updates / (ms * 1e-3), "unit": "updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "knn200k", "N": n, "nnz_off": nnz, "R": eta, "p": p, "k_nn": wl["knn"],
                   "sigma": wl["sigma"], "step": "filter + backward (edge weights, coefficients)",
                   "sweeps_per_step": 3,
                   "l2": "inputs smaller than L2: a 256 MB buffer is overwritten between timed steps"},
        "gpu_launches": launches, "roofline": roof, "roofline_by_variant": by_variant, "clocks": clocks,
        "e2e": None,
        "gradient_check": {"directional_fd": fd, "adjoint": an, "rel_diff": abs(fd - an) / max(abs(fd), 1e-300),
                           "h": h},
        "clustering": cluster_recovery(sf, g, lh, R, wl["k"], p, labels, seed=wl["r_seed"]),
        "stability": stability_leg(sf, g, lh, p, n, eta, wl["k"], seed=wl["r_seed"]),
    }
    g.free()
    return out


def adjusted_rand_index(a, b):
    """Adjusted Rand index of two labelings (Hubert and Arabie, 1985)."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1), np.int64)
    np.add.at(table, (ai, bi), 1)
    comb = lambda x: x * (x - 1) / 2.0  # noqa: E731
    s_ij = comb(table).sum()
    s_a = comb(table.sum(1)).sum()
    s_b = comb(table.sum(0)).sum()
    expected = s_a * s_b / comb(len(a))
    top = 0.5 * (s_a + s_b)
    return float((s_ij - expected) / (top - expected)) if top != expected else 1.0


def stability_leg(sf, g, lh, p, n, eta, k, seed, J=4, half_width=2, starts=4):
    """gamma(k) of §4.3 / Eq. (12) around the generating k, J realisations: at the
    order that separates the filters of adjacent k (p_filter = 0) and, beside it,
    with the filters at the count's order p."""
    import torch

    from paper_1509_08863_gb300 import synth

    Rc = torch.as_tensor(synth.gaussian_block(n, eta, seed + 101), dtype=torch.float32, device="cuda")
    R = torch.as_tensor(np.stack([synth.gaussian_block(n, eta, seed + 200 + j) for j in range(J)]),
                        dtype=torch.float32, device="cuda")
    kmin, kmax = max(2, k - half_width), k + half_width
    ks = list(range(kmin, kmax + 1))
    out = {"k": ks, "generating_k": k, "realisations": J, "starts": starts, "count_order": p}
    for name, pf in (("resolving_order", 0), ("count_order", None)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gamma, lam_k, used = sf.stability(g, lh, p, Rc, R, kmin, kmax, 50, starts, seed, p_filter=pf,
                                          return_order=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"filter_order": used, "gamma": [float(x) for x in gamma], "lam_k": [float(x) for x in lam_k],
                     "k_star": ks[int(np.argmax(gamma))], "ms": e0.elapsed_time(e1)}
    out.update(out["resolving_order"])
    return out


def cluster_recovery(sf, g, lh, R, k, p, truth, seed, restarts=10):
    """§4.1 end to end on the graph: eigencount for lambda_k (count k - 1/2),
    filter R at it, row-normalised features, k-means with several seeded
    restarts (the lowest inertia kept); the adjusted Rand index against the
    generating labels."""
    import torch

    n = R.shape[0]
    mu = sf.cheb_moments(g, lh, R, p)
    lk = sf.dichotomy(mu, p, lh, k - 0.5)
    a = sf.cheb_coeffs(lh, lk, p, True)
    F = sf.features(sf.cheb_filter(g, lh, a, R)[0], True)
    rng = np.random.default_rng(seed)
    best = None
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(restarts):
        C0 = F[torch.as_tensor(rng.choice(n, k, replace=False), device=F.device)].contiguous()
        lab, _, it, inertia = sf.kmeans(F, C0, 100)
        if best is None or inertia < best[1]:
            best = (lab, inertia, it)
    e1.record()
    torch.cuda.synchronize()
    return {"k": k, "lam_k_estimate": lk, "restarts": restarts, "kmeans_ms_total": e0.elapsed_time(e1),
            "best_inertia": best[1], "assignments_of_best": best[2],
            "ari_vs_generating_labels": adjusted_rand_index(best[0].cpu().numpy(), truth)}


def run_batch(args, wl):
    """256 graphs of uneven size filtered with per-graph cutoffs: one sweep
    launch per order for the whole batch, against one filter call per graph."""
    import torch

    import paper_1509_08863_gb300 as sf
    from paper_1509_08863_gb300 import build as sfbuild
    from paper_1509_08863_gb300 import synth

    sfbuild.build()
    dev = torch.device("cuda")
    eta, p = wl["R"], wl["p"]
    st = sf.BF16 if wl["storage"] == "bf16" else sf.F32
    graphs, ks = synth.batched_sbm(wl["n_graphs"], wl["graph_seed"])
    gs, lams, cuts = [], [], []
    for gr, kk in zip(graphs, ks):
        g = sf.csr_build(gr.n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
        _, lh = sf.lambda_max_estimate(g, 40, None, seed=11)
        gs.append(g)
        lams.append(lh)
    b = sf.batch_build(gs)
    n_tot, nnz_tot, ng, offs = b.info()
    R_host = synth.gaussian_block(n_tot, eta, wl["r_seed"])
    R = torch.as_tensor(R_host, dtype=torch.float32, device=dev)
    # per-graph cutoff: the dichotomy for that graph's community count (setup, untimed)
    coeffs = np.zeros((ng, p + 1))
    for i in range(ng):
        sl = slice(int(offs[i]), int(offs[i + 1]))
        mu = sf.cheb_moments(gs[i], lams[i], R[sl].contiguous(), p)
        lk = sf.dichotomy(mu, p, lams[i], float(ks[i]) - 0.5)
        cuts.append(lk)
        coeffs[i] = sf.cheb_coeffs(lams[i], lk, p, True)[0]
    tuned = sf.autotune(gs[int(np.argmax(np.diff(offs)))], eta, st, 1)
    opts = sf.Opts(storage=st, slab_cols=tuned.slab_cols, block_warps=tuned.block_warps,
                   carveout_pct=tuned.carveout_pct, l2_window=tuned.l2_window, sweep_kernel=tuned.sweep_kernel)
    Y = torch.empty((n_tot, eta), dtype=torch.float32, device=dev)
    Rs = [R[int(offs[i]):int(offs[i + 1])].contiguous() for i in range(ng)]
    Ys = [torch.empty_like(x) for x in Rs]

    def batched():
        sf.cheb_filter_batched(b, np.array(lams), coeffs, R, opts, out=Y)

    def sequential():
        for i in range(ng):
            sf.cheb_filter(gs[i], lams[i], coeffs[i][None, :], Rs[i], opts, out=Ys[i][None])

    ms_b, launches_b, variants_b, clocks = _clock_timed(batched, args.steps, args.warmup, sf)
    # the same call with device tables, captured once into a CUDA graph and replayed
    tol_d = torch.as_tensor(2.0 / np.array(lams), dtype=torch.float64, device=dev)
    coef_d = torch.as_tensor(coeffs, dtype=torch.float32, device=dev)
    Yg = torch.empty_like(Y)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Yg, opts)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Yg, opts)
    ms_g, launches_g, _, _ = _clock_timed(cg.replay, args.steps, 1, sf)
    graph_same = bool(torch.equal(Yg, Y))
    # the same batch in one persistent launch for all orders (per-graph arrival counters), eager and captured;
    # its shape is the staged-tile kernel's (8 warps, 40% carveout: its fastest on this batch)
    opts_p = sf.Opts(storage=st, slab_cols=tuned.slab_cols, block_warps=8, carveout_pct=40,
                     sweep_kernel=sf.SWEEP_PERSISTENT)
    Yp = torch.empty_like(Y)

    def persistent():
        sf.cheb_filter_batched(b, np.array(lams), coeffs, R, opts_p, out=Yp)

    ms_p, launches_p, variants_p, _ = _clock_timed(persistent, args.steps, 1, sf)
    Ypg = torch.empty_like(Y)
    with torch.cuda.stream(side):
        sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Ypg, opts_p)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    cgp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cgp):
        sf.cheb_filter_batched_dev(b, tol_d, coef_d, R, Ypg, opts_p)
    ms_pg, _, _, _ = _clock_timed(cgp.replay, args.steps, 1, sf)
    ms_s, launches_s, _, _ = _clock_timed(sequential, max(1, args.steps // 2), 1, sf)
    nnz_sum = sum(g.nnz for g in gs)
    updates = (nnz_sum + n_tot) * eta * p
    roof, by_variant = _roof_variants(variants_b, args.workload)
    # the two forms compute the same rows bit for bit
    same = all(torch.equal(Y[int(offs[i]):int(offs[i + 1])], Ys[i]) for i in range(ng))
    out = {
        "metric": "filtered nnz*R*p updates/s", "value": updates / (ms_b * 1e-3), "unit": "updates/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": f"{wl['storage']}-storage/f32-compute",
        "data": "synthetic",
        "config": {"workload": "batch256", "graphs": ng, "N_total": n_tot, "nnz_off_total": nnz_sum, "R": eta,
                   "p": p, "block_storage": wl["storage"], "tiles": {"slab_cols": tuned.slab_cols,
                                                                     "block_warps": tuned.block_warps,
                                                                     "sweep_kernel": ("auto", "tiled", "direct")[
                                                                         tuned.sweep_kernel]},
                   "l2": "inputs larger than L2 (no flush)"},
        "gpu_launches": launches_b, "roofline": roof, "roofline_by_variant": by_variant, "clocks": clocks,
        "e2e": None,
        "sequential": {"value": updates / (ms_s * 1e-3), "ms_per_step": ms_s, "gpu_launches": launches_s,
                       "speedup_of_batching": ms_s / ms_b},
        "batched_equals_sequential": bool(same),
        "cuda_graph": {"value": updates / (ms_g * 1e-3), "ms_per_step": ms_g, "equals_eager": graph_same,
                       "note": "one capture of the device-table batched call, replayed"},
        "persistent": {"value": updates / (ms_p * 1e-3), "ms_per_step": ms_p, "gpu_launches": launches_p,
                       "equals_per_order": bool(torch.equal(Yp, Y)),
                       "cuda_graph_ms_per_step": ms_pg, "cuda_graph_equals": bool(torch.equal(Ypg, Y)),
                       "roofline_by_variant": _roof_variants(variants_p, args.workload)[1],
                       "note": "one launch per column slab runs all orders: blocks claim (order, 8-tile chunk) items "
                               "and wait on per-graph arrival counters"},
    }
    out.update(batch_fp32_and_accuracy(sf, b, gs, lams, coeffs, R, Rs, Y, offs, opts, updates, ms_b, args, graphs,
                                       ks, R_host))
    for g in gs:
        g.free()
    b.free()
    return out


def config_sbm1k(sf, args):
    """The small parity workload: FP32 filter at p = 50 on the 1000-node SBM with
    the cutoff at the true lambda_k (dense eigendecomposition of L), its time
    and its error against the FP64 oracle (all columns)."""
    import torch

    import oracle

    wl = WORKLOADS["sbm1k"]
    dev = torch.device("cuda")
    gr, R = make_inputs(wl)
    n, p, k = wl["n"], wl["p"], wl["k"]
    g = sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    go = oracle.csr_build(n, gr.src, gr.dst, gr.w)
    Wd = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(go.rowptr))
    Wd[rows, go.colidx] = go.val
    lam_true = np.linalg.eigvalsh(np.diag(Wd.sum(1)) - Wd)
    # lam_hat from the oracle's Lanczos: the same input on both sides
    lh = oracle.lambda_hat(oracle.lanczos_max(go, 60, np.random.default_rng(1).standard_normal(n)),
                           oracle.strength(go))
    a = oracle.cheb_coeffs(lh, float(lam_true[k - 1]), p, True)
    Rt = torch.as_tensor(R, dtype=torch.float32, device=dev)
    Y = torch.empty((1, n, wl["R"]), dtype=torch.float32, device=dev)
    ms, launches, variants, _ = _clock_timed(lambda: sf.cheb_filter(g, lh, a, Rt, None, out=Y), 20, 3, sf,
                                             flush_l2=True)
    Yo = oracle.cheb_filter(go, lh, a, R)[0]
    err = float(np.linalg.norm(Y[0].cpu().numpy() - Yo) / np.linalg.norm(Yo))
    roof, _ = _roof_variants(variants, "sbm1k")
    g.free()
    return {"N": n, "nnz_off": go.nnz, "R": wl["R"], "p": p, "storage": "f32", "cutoff": "true lambda_k",
            "ms_per_filter": ms, "updates_per_s": (go.nnz + n) * wl["R"] * p / (ms * 1e-3),
            "rel_fro_error_vs_fp64_oracle": err, "tolerance": 1e-5, "within_tolerance": err <= 1e-5,
            "gpu_launches_per_filter": launches / 20, "roofline": roof,
            "note": "working set (0.4 MB) lives in L2: a launch-latency-bound case, not an HBM roofline one"}


def config_sbm100k(sf, args):
    """The eigenvalue count of §3.2 on the 100k-node SBM: one FP32 moment sweep
    (p = 100) gives the counts at 16 cutoffs uniform in [0, 0.2 lam_hat]; its
    time, roofline and the moments against the FP64 oracle on 2 columns."""
    import torch

    import oracle

    wl = WORKLOADS["sbm100k"]
    dev = torch.device("cuda")
    gr, R = make_inputs(wl)
    n, p = wl["n"], wl["p"]
    g = sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    _, lh = sf.lambda_max_estimate(g, 40, None, seed=11)
    Rt = torch.as_tensor(R, dtype=torch.float32, device=dev)
    cuts = np.linspace(0.0, 0.2 * lh, 16)
    holder = {}

    def sweep():
        holder["mu"] = sf.cheb_moments(g, lh, Rt, p)

    ms, launches, variants, _ = _clock_timed(sweep, 10, 3, sf, flush_l2=True)
    counts = sf.eigencount_from(holder["mu"], p, lh, cuts)
    roof, by_variant = _roof_variants(variants, "sbm100k")
    go = oracle.csr_build(n, gr.src, gr.dst, gr.w)
    R2 = np.ascontiguousarray(R[:, :2])
    lo = oracle.lambda_hat(oracle.lanczos_max(go, 40, np.random.default_rng(2).standard_normal(n)),
                           oracle.strength(go))  # the oracle's lam_hat, given to both sides
    mu2 = sf.cheb_moments(g, lo, torch.as_tensor(R2, dtype=torch.float32, device=dev), p)
    muo = oracle.moments(go, lo, R2, 2 * p)
    worst = float(np.max(np.abs(mu2 - muo) / ((np.arange(2 * p + 1) + 1) * muo[0])))
    nnz = g.nnz
    g.free()
    return {"N": n, "nnz_off": nnz, "R": wl["R"], "p": p, "storage": "f32", "cutoffs": cuts.tolist(),
            "counts": counts.tolist(), "ms_per_sweep": ms, "updates_per_s": (nnz + n) * wl["R"] * p / (ms * 1e-3),
            "gpu_launches_per_sweep": launches / 10, "roofline": roof, "roofline_by_variant": by_variant,
            "moments_vs_fp64_oracle_2_columns": {"max_err_over_(m+1)mu0": worst, "tolerance": 2e-6,
                                                 "within_tolerance": worst <= 2e-6},
            "note": "the graph and one 64-column block (34 MB) fit in L2: after the first order the sweep runs "
                    "from L2, so its HBM fraction is not a DRAM-bound figure"}


def other_configs(args, sf):
    """The other workloads, each as a sub-object of the default run's JSON line."""
    import copy

    out = {}
    sub = copy.copy(args)
    sub.steps, sub.warmup = max(3, args.steps // 4), 3
    for name, fn in (("sbm1k", lambda: config_sbm1k(sf, sub)), ("sbm100k", lambda: config_sbm100k(sf, sub)),
                     ("knn200k", lambda: run_knn_grad(sub, WORKLOADS["knn200k"])),
                     ("batch256", lambda: run_batch(sub, WORKLOADS["batch256"]))):
        sub.workload = name  # each leg reads its own workload's profile figures
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:  # one leg failing must not lose the others
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def batch_fp32_and_accuracy(sf, b, gs, lams, coeffs, R, Rs, Y, offs, opts, updates, ms_b, args, graphs, ks,
                            R_host):
    """The batch with plain FP32 blocks (batched and sequential: the plain form),
    and the feature accuracy of the BF16 batch against FP32 and, on two small
    graphs, against the FP64 oracle."""
    import torch

    import oracle

    ng = len(gs)
    o32 = sf.Opts(storage=sf.F32, algo=sf.ALGO_FORWARD)
    Y32 = torch.empty_like(Y)
    Ys32 = [torch.empty_like(x) for x in Rs]

    def batched32():
        sf.cheb_filter_batched(b, np.array(lams), coeffs, R, o32, out=Y32)

    def sequential32():
        for i in range(ng):
            sf.cheb_filter(gs[i], lams[i], coeffs[i][None, :], Rs[i], o32, out=Ys32[i][None])

    ms_b32, _, _, _ = _clock_timed(batched32, max(1, args.steps // 2), 1, sf)
    ms_s32, _, _, _ = _clock_timed(sequential32, max(1, args.steps // 2), 1, sf)
    F16 = sf.features(Y, True).cpu().numpy().astype(np.float64)
    F32 = sf.features(Y32, True).cpu().numpy().astype(np.float64)
    ce = row_cosine_error(F16, F32)
    # the FP64 oracle on the two smallest graphs: lam_hat from its Lanczos, the cutoff at the graph's
    # k-th eigenvalue from a dense eigendecomposition (host), both forms as single-graph calls with these
    # inputs (the batched call equals them bit for bit, checked above)
    orc = {}
    p = coeffs.shape[1] - 1
    for i in np.argsort(np.diff(offs))[:2]:
        i = int(i)
        gr, kk = graphs[i], int(ks[i])
        go = oracle.csr_build(gr.n, gr.src, gr.dst, gr.w)
        s_o = oracle.strength(go)
        lh_o = oracle.lambda_hat(oracle.lanczos_max(go, 60, np.random.default_rng(i).standard_normal(gr.n)), s_o)
        Wd = np.zeros((gr.n, gr.n))
        Wd[np.repeat(np.arange(gr.n), np.diff(go.rowptr)), go.colidx] = go.val
        lam = np.linalg.eigvalsh(np.diag(Wd.sum(1)) - Wd)
        a_o = oracle.cheb_coeffs(lh_o, 0.5 * (lam[kk - 1] + lam[kk]), p, True)
        Ri = R_host[int(offs[i]):int(offs[i + 1])]
        Fo = oracle.features(oracle.cheb_filter(go, lh_o, a_o, Ri)[0], True)
        Rg = torch.as_tensor(Ri, dtype=torch.float32, device="cuda")
        res = {}
        for name, st in (("bf16", sf.BF16), ("f32", sf.F32)):
            Fg = sf.features(sf.cheb_filter(gs[i], lh_o, a_o, Rg, sf.Opts(storage=st, algo=sf.ALGO_FORWARD))[0],
                             True).cpu().numpy().astype(np.float64)
            ce_i = row_cosine_error(Fg, Fo)
            res[name] = {"median": float(np.median(ce_i)), "max": float(ce_i.max())}
        orc[f"graph_{i}_N{gr.n}_k{kk}"] = res
    return {
        "fp32_batched": {"value": updates / (ms_b32 * 1e-3), "ms_per_step": ms_b32},
        "fp32_sequential": {"value": updates / (ms_s32 * 1e-3), "ms_per_step": ms_s32,
                            "note": "the plain form: one FP32-block filter call per graph"},
        "speedup_vs_plain_fp32": ms_s32 / ms_b,
        "feature_accuracy": {"bf16_vs_f32_cosine_error": {"median": float(np.median(ce)),
                                                          "p99": float(np.quantile(ce, 0.99)),
                                                          "max": float(ce.max())},
                             "vs_fp64_oracle_cosine_error": orc},
    }


# the accuracy legs' cutoff as a fraction of lam_hat (the 1M-node SBM's lambda_k / lam_hat is about 0.18)
CUTOFF_OVER_LAM_HAT = 0.18


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def row_cosine_error(A, B):
    """Per-row 1 - cos(A_i, B_i) (rows of two feature blocks)."""
    na = np.linalg.norm(A, axis=1)
    nb = np.linalg.norm(B, axis=1)
    ok = (na > 0) & (nb > 0)
    c = np.einsum("ij,ij->i", A[ok], B[ok]) / (na[ok] * nb[ok])
    return np.clip(1.0 - c, 0.0, None)


def cpu_baseline_and_accuracy(gr, R, info, wl, sf, dev, cols=8, serial_orders=24):
    """The FP64 oracle on `cols` of the block's signal columns (all N nodes):
    (ii) the OpenMP build on every host core at the full order p -- the CPU
    baseline, whose output also measures the GPU filter's error on those
    columns -- and (i) the plain single-thread build on the same columns for
    `serial_orders` orders (bounded time). Both builds give identical results."""
    import torch

    import oracle

    n, p = wl["n"], wl["p"]
    g = oracle.csr_build(n, gr.src, gr.dst, gr.w)
    # lam_hat from the oracle's own Lanczos (40 steps, seeded start) and the cutoff at a
    # stated fraction of it, near the workload's lambda_k: both sides get these inputs
    v0 = np.random.default_rng(wl["graph_seed"] + 17).standard_normal(n)
    lh = oracle.lambda_hat(oracle.lanczos_max(g, 40, v0), oracle.strength(g))
    lk = CUTOFF_OVER_LAM_HAT * lh
    a = oracle.cheb_coeffs(lh, lk, p, True)
    Rs = np.ascontiguousarray(R[:, :cols])
    cores = host_cores()
    legs = {}
    Yo = None
    try:
        oracle.build_parallel()
        thr = oracle.threads(parallel=True)
        t0 = time.perf_counter()
        Yo = oracle.cheb_filter(g, lh, a, Rs, parallel=True)[0]
        dt = time.perf_counter() - t0
        legs["all_cores"] = {"value": (g.nnz + n) * cols * p / dt, "unit": "updates/s", "threads": thr,
                             "seconds": dt, "sample": f"{cols} of {wl['R']} signal columns, all {n} nodes, p={p}"}
    except Exception as e:
        legs["all_cores"] = {"unavailable": f"OpenMP build of the oracle failed: {e}"}
    p1 = min(p, serial_orders)
    a1 = oracle.cheb_coeffs(lh, lk, p1, True)
    t0 = time.perf_counter()
    oracle.cheb_filter(g, lh, a1, Rs)
    dt1 = time.perf_counter() - t0
    legs["one_thread"] = {"value": (g.nnz + n) * cols * p1 / dt1, "unit": "updates/s", "threads": 1,
                          "seconds": dt1, "sample": f"{cols} of {wl['R']} signal columns, all {n} nodes, "
                                                    f"{p1} of the {p} orders"}
    if Yo is None:  # no OpenMP: the accuracy reference comes from the plain build
        Yo = oracle.cheb_filter(g, lh, a, Rs)[0]
    main = legs["all_cores"] if "value" in legs["all_cores"] else legs["one_thread"]
    cpu = {"value": main["value"], "unit": "updates/s", "cores": main["threads"], "host_cores": cores,
           "kind": "oracle", "sample": main["sample"] + " (oracle_cheb_filter, FP64)", "legs": legs}
    # GPU filter outputs on the same columns (run on the whole block, as in the step)
    gg = sf.csr_build(n, torch.as_tensor(gr.src, device=dev), torch.as_tensor(gr.dst, device=dev), None)
    Rt = torch.as_tensor(R, dtype=torch.float32, device=dev)
    acc = {}
    rows = np.random.default_rng(5).choice(n, size=min(50_000, n), replace=False)
    Fo = Yo[rows] / np.linalg.norm(Yo[rows], axis=1, keepdims=True)
    feats = {}
    for name, st, algo in (("f32", sf.F32, sf.ALGO_CLENSHAW), ("bf16", sf.BF16, sf.ALGO_FORWARD),
                           ("f16", sf.F16, sf.ALGO_FORWARD), ("f32_forward", sf.F32, sf.ALGO_FORWARD),
                           ("bf16_clenshaw", sf.BF16, sf.ALGO_CLENSHAW), ("f16_clenshaw", sf.F16, sf.ALGO_CLENSHAW)):
        Yfull = sf.cheb_filter(gg, lh, a, Rt, sf.Opts(storage=st, algo=algo))[0]
        Y = Yfull[:, :cols].cpu().numpy().astype(np.float64)
        ce = row_cosine_error(Y[rows], Fo)
        acc[name] = {
            "rel_fro_all_rows": float(np.linalg.norm(Y - Yo) / np.linalg.norm(Yo)),
            "rel_fro_50k_rows": float(np.linalg.norm(Y[rows] - Yo[rows]) / np.linalg.norm(Yo[rows])),
            "feature_cosine_error_50k_rows": {"median": float(np.median(ce)), "p99": float(np.quantile(ce, 0.99)),
                                              "max": float(ce.max())},
        }
        if name in ("f32", "bf16", "f16"):
            feats[name] = sf.features(Yfull, True)
        del Yfull
    acc["features_note"] = (f"features of Eq. (11) restricted to the {cols} oracle columns: each GPU row's first "
                            f"{cols} filtered values against the FP64 oracle's, normalised, on 50,000 sampled rows")
    # k-means labels from the 16-bit features against those from FP32 features (identical starts)
    k = wl["k"]
    start = torch.as_tensor(np.random.default_rng(wl["r_seed"] + 9).choice(n, k, replace=False), device=dev)
    labs = {}
    for name, F in feats.items():
        lab, _, it, _ = sf.kmeans(F, F[start].contiguous().clone(), 30)
        labs[name] = lab.cpu().numpy()
    acc["kmeans_labels_vs_f32"] = {name: {"ari": adjusted_rand_index(labs[name], labs["f32"]),
                                          "equal_fraction": float(np.mean(labs[name] == labs["f32"]))}
                                   for name in ("bf16", "f16")}
    acc["kmeans_note"] = (f"k = {k}, 30 Lloyd iterations from the same {k} rows of each feature block (all "
                          f"{wl['R']} columns, all rows)")
    # moments in BF16 blocks vs FP32 blocks: effect on the counts and on the dichotomy
    mu32 = sf.cheb_moments(gg, lh, Rt, p, sf.Opts(storage=sf.F32))
    mu16 = sf.cheb_moments(gg, lh, Rt, p, sf.Opts(storage=sf.BF16))
    cuts = np.array([0.5, 0.8, 1.0, 1.25, 2.0]) * lk
    acc["moments"] = {
        "cutoffs_over_lam_k": [0.5, 0.8, 1.0, 1.25, 2.0],
        "counts_f32_blocks": sf.eigencount_from(mu32, p, lh, cuts).tolist(),
        "counts_bf16_blocks": sf.eigencount_from(mu16, p, lh, cuts).tolist(),
        "lam_k_f32_blocks": sf.dichotomy(mu32, p, lh, wl["k"] - 0.5),
        "lam_k_bf16_blocks": sf.dichotomy(mu16, p, lh, wl["k"] - 0.5),
    }
    del feats
    gg.free()
    acc["reference"] = (f"FP64 oracle, columns 0..{cols - 1}; lam_hat {lh:.6g} from the oracle's Lanczos, cutoff "
                        f"{CUTOFF_OVER_LAM_HAT} lam_hat, the same coefficients on both sides")
    return cpu, acc


if __name__ == "__main__":
    sys.exit(main())
