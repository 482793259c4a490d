"""Benchmark of the layered-media FMM on one or more GB300s.

One step = one pass of the whole hot path on one synthetic charge set that is
already resident in HBM: octree build (classify, Morton sort, boxes,
interaction lists) followed by the evaluation of potentials and fields
(P2M, M2M, free-space and reaction M2L, L2L, L2P, near field, component
sum).  Workload: three-layer medium (interfaces z=0, z=-1.2, eps=(1,5,10)),
N = 1,048,576 charges split equally between the layers, p = 10, leaf
capacity 40.  ``value`` is particles/s of the headline form: FP32 P2P, M2L
and L2P with compensated sums, FP64 Sommerfeld tables, and the learned
near-field reaction kernels switched on (their one-off training per medium
runs before the timed region and is reported as ``surrogate_train_s``).  The
FP32 form without the network and the plain FP64 form are timed on the same
input and reported beside it.  In this workload no reaction pair is close
enough to reach the near field, so the network is idle here; a second,
near-interface workload (every charge within 0.02 of an interface) measures
what it gains there (``near_interface``).

With --gpus N (torchrun, one process per GPU) every rank runs an independent
replica of the step (the method needs no exchange between GPUs for one
problem); ``value`` is all particles processed / the slowest rank's time.

``--impl reference`` times the CPU oracle (direct FP64 sum, exact
three-layer image series) on the host cores on a bounded sample of targets
of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s at N=1M p=10 (FP32+surrogate vs plain FP64 GPU), rel L2 err"
FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 of a GB300 (no measured figure available)
SMS = 152


def fp32_peak_tflops(sm_mhz):
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return SMS * 128 * 2 * sm_mhz * 1e6 / 1e12


# Dense TF32 tensor peak: the measured bf16 GEMM rate of the GB300s
# times the nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s); fallback 1.9 PF bf16.
TF32_PER_BF16 = 1.1 / 2.25
# DRAM bytes (read + write) of one k_m2l_tc launch per free-space M2L pair,
# from an ncu capture of the bench's own workload (N=1,048,576, p=10: 245.1 MB
# read + 33.3 MB written for 10,905,072 pairs), scaled to the bench's pair count.
TC_DRAM_BYTES_PER_PAIR = (245.149952e6 + 33.294592e6) / 10905072


def tf32_peak_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16 = float(json.load(fh)["bf16_tflops"])
        src = "of measured"
    except Exception:
        bf16, src = 1900.0, "of fallback"
    return bf16 * TF32_PER_BF16, src


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--p", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 leg")
    ap.add_argument("--sample", type=int, default=256, help="oracle targets for the accuracy / CPU leg")
    ap.add_argument("--no-near", action="store_true", help="skip the near-interface workload")
    ap.add_argument("--no-multi", action="store_true", help="skip the many-charge-vector workload")
    ap.add_argument("--no-batch", action="store_true", help="skip the many-problem workload")
    ap.add_argument("--no-four", action="store_true", help="skip the four-layer workload")
    ap.add_argument("--acc-targets", default="200,60",
                    help="oracle targets of the two N = 1M cases of --accuracy-table")
    ap.add_argument("--accuracy-table", action="store_true",
                    help="instead of timing: Err2 against the oracle for each medium, N, p and precision")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the headline: time and Err2 for N in {64k, 256k, 1M} x p in {6, 10, 14} x form")
    ap.add_argument("--matched-orders", default="8,9",
                    help="orders of the plain FP64 form timed beside the headline for the matched-accuracy line")
    ap.add_argument("--forms", default="fp32_surrogate,fp32,fp64",
                    help="comma list of fp32_surrogate, fp32, fp64; the first is the headline")
    return ap.parse_args()


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples go to BENCH_CLOCKS_DIR (if set) or the temporary directory
        d = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, "lfmm_clocks_rank%d_%d.csv" % (index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allmax(pg, v):
    if pg is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def oracle_sample(w, count):
    import oracle
    from paper_1908_10863_gb300 import workloads
    t = workloads.subsample(w.n, count)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES,
                              threads=threads)
    dt = time.perf_counter() - t0
    return t, ref, refE, dt, threads


def err2_per_layer(ref, got, layers):
    """Err2 of Section 4 over the sampled targets of each layer, keyed by layer id."""
    import oracle
    layers = np.asarray(layers)
    return {str(int(l)): oracle.err2(ref[layers == l], got[layers == l]) for l in np.unique(layers)}


def form_label(name, st):
    """What the headline form ran, from the build and evaluation statistics:
    the learned near-field kernels are only named as used when they
    evaluated pairs."""
    base = {"fp32_surrogate": "FP32 P2P/M2L/L2P, compensated sums, FP64 Sommerfeld tables",
            "fp32": "FP32 P2P/M2L/L2P, compensated sums, FP64 Sommerfeld tables",
            "fp64": "FP64 throughout"}[name]
    if name != "fp32_surrogate":
        return base
    net, quad = int(st.get("surr_net_pairs", 0)), int(st.get("surr_quad_pairs", 0))
    if net == 0:
        return (base + "; learned near-field reaction kernels enabled but idle: the near field holds no reaction "
                "pairs at this size (network pairs 0, quadrature pairs %d), so this is the plain FP32 form; the "
                "network's effect is measured on the near-interface workload" % quad)
    return base + "; learned near-field reaction kernels on (network pairs %d, quadrature pairs %d)" % (net, quad)


def m2l_flops_per_pair(p):
    # dense M2L: (p+1)^2 source coefficients x (p+1)(p+2)/2 target coefficients, complex MAC = 8 flops
    return 8 * (p + 1) ** 2 * (p + 1) * (p + 2) // 2


SURR_SAMPLES, SURR_EPOCHS, SURR_SEED = 1 << 18, 32, 5


def run_form(f, xyz_d, lay_d, q_d, phi_d, fld_d, torch, steps, warmup, flush):
    """W untimed then K timed steps; stage times come from the library's own
    CUDA events on the launching stream, recorded inside the timed steps."""
    stream = torch.cuda.current_stream()

    def step():
        f.build_device(xyz_d, lay_d, stream)
        f.evaluate_device(q_d, phi_d, fld_d, stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches0 = f.stats()["launches"]
    f.set_option(3, 1)  # stage events
    times, stages = [], []
    for _ in range(steps):
        flush.fill_(1.0)  # evict L2 between steps (untimed)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        stages.append(f.timings())
    f.set_option(3, 0)
    torch.cuda.synchronize()
    launches = f.stats()["launches"] - launches0
    mean = {k: sum(s_[k] for s_ in stages) / len(stages) for k in stages[0]}
    return times, launches, mean


def near_interface_leg(torch, dev, p, flush):
    """P2P stage and whole step on the near-interface workload: quadrature vs network."""
    from paper_1908_10863_gb300 import LayeredFMM, workloads
    import oracle
    w = workloads.near_interface(1 << 18)
    xyz_d = torch.from_numpy(w.xyz).to(dev)
    lay_d = torch.from_numpy(w.layer).to(dev)
    q_d = torch.from_numpy(w.q).to(dev)
    phi_d = torch.empty(w.n, dtype=torch.float64, device=dev)
    fld_d = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
    out = {"workload": "three-layer medium d=(0,-1.2) eps=(1,5,10), N=%d charges within 0.02 of an interface, "
                       "q~U[-1,1], p=%d, leaf 40" % (w.n, p)}
    for prec, pname in ((0, "fp64"), (1, "fp32")):
        f = LayeredFMM(w.d, w.eps, p, precision=prec)
        f.surrogate_train(SURR_SAMPLES, SURR_EPOCHS, SURR_SEED)
        table_err = f.near_tables()
        phis = {}
        # near-field reaction kernels by quadrature, by the network, by the pre-computed tables
        for kind, surr, tab in (("quadrature", 0, 0), ("network", 1, 0), ("tables", 0, 1)):
            f.set_option(5, surr)
            f.set_option(10, tab)
            times, launches, stages = run_form(f, xyz_d, lay_d, q_d, phi_d, fld_d, torch, 2, 1, flush)
            st = f.stats()
            out[pname + "_" + kind] = {"ms_per_step": sum(times) / len(times), "p2p_ms": stages["p2p"],
                                       "pairs_network": st["surr_net_pairs"], "pairs_quadrature": st["surr_quad_pairs"]}
            phis[kind] = phi_d.cpu().numpy().copy()
        f.set_option(10, 0)
        for kind in ("network", "tables"):
            out[pname + "_" + kind]["err2_phi_vs_quadrature"] = oracle.err2(phis["quadrature"], phis[kind])
            out[pname + "_" + kind + "_p2p_speedup"] = (out[pname + "_quadrature"]["p2p_ms"] /
                                                        out[pname + "_" + kind]["p2p_ms"])
        out[pname + "_tables"]["table_max_rel_err"] = table_err
        f.close()
    return out


def four_layer_leg(torch, dev, p, flush, n=1 << 20, targets=48):
    """Media of four layers at N = 1M: interfaces (0, -0.6, -1.2), both forms
    timed on eps = (2, 7, 1.5, 12); accuracy on eps = (1, 5, 5, 10), whose
    middle interface separates equal permittivities, against the exact
    three-layer image series (the oracle's quadrature is too slow at 1M)."""
    from paper_1908_10863_gb300 import LayeredFMM, workloads
    import oracle
    out = {"workload": "four-layer medium d=(0,-0.6,-1.2), N=%d charges split equally between layers, q~U[-1,1], "
                       "p=%d, leaf 40" % (n, p)}
    for eps, tag in ((workloads.EPS_FOUR, "timed"), ((1.0, 5.0, 5.0, 10.0), "merged")):
        w = workloads.four_layers(n, eps=eps)
        xyz_d = torch.from_numpy(w.xyz).to(dev)
        lay_d = torch.from_numpy(w.layer).to(dev)
        q_d = torch.from_numpy(w.q).to(dev)
        phi_d = torch.empty(w.n, dtype=torch.float64, device=dev)
        fld_d = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
        for prec, pname in ((1, "fp32"), (0, "fp64")):
            if tag == "merged" and prec == 0:
                continue
            f = LayeredFMM(w.d, w.eps, p, precision=prec)
            steps = 3 if prec else 2
            times, launches, stages = run_form(f, xyz_d, lay_d, q_d, phi_d, fld_d, torch, steps, 1, flush)
            st = f.stats()
            f.close()
            ms = sum(times) / len(times)
            if tag == "timed":
                out[pname] = {"ms_per_step": ms, "particles_per_s": w.n / (ms / 1e3),
                              "stage_ms": stages, "components": st["components"],
                              "m2l_reaction": st["m2l_reaction"], "p2p_reaction": st["p2p_reaction"],
                              "reaction_tables": st["reaction_tables"]}
            else:
                t = workloads.subsample(w.n, targets)
                lay3 = np.where(w.layer >= 2, w.layer - 1, w.layer).astype(np.int32)
                ref, refE = oracle.direct([0.0, -1.2], [1.0, 5.0, 10.0], w.xyz, lay3, w.q, targets=t,
                                          mode=oracle.MODE_IMAGES)
                phi = phi_d.cpu().numpy()
                fld = fld_d.cpu().numpy()
                out["merged_fp32"] = {"ms_per_step": ms, "err2_phi": oracle.err2(ref, phi[t]),
                                      "err2_field": oracle.err2(refE, fld[t]), "targets": int(len(t))}
    return out


def multi_rhs_leg(torch, dev, p, flush, nrhs=64, n=1 << 18):
    """Float32 form, one tree, nrhs charge vectors: one batched call against
    nrhs single calls (device buffers, CUDA events)."""
    from paper_1908_10863_gb300 import LayeredFMM, workloads
    w = workloads.config2(n)
    Q = np.random.default_rng(workloads.SEED_BASE + 5).uniform(-1.0, 1.0, (nrhs, w.n))
    q_d = torch.from_numpy(Q).to(dev)
    phi_d = torch.empty_like(q_d)
    fld_d = torch.empty((nrhs, w.n, 3), dtype=torch.float64, device=dev)
    f = LayeredFMM(w.d, w.eps, p, precision=1)
    xyz_d = torch.from_numpy(w.xyz).to(dev)
    lay_d = torch.from_numpy(w.layer).to(dev)
    s = torch.cuda.current_stream()
    f.build_device(xyz_d, lay_d, s)

    def timed(fn):
        fn()  # warm-up
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        return a.elapsed_time(b)

    t_batch = timed(lambda: f.evaluate_device(q_d, phi_d, fld_d, s))
    t_single = timed(lambda: [f.evaluate_device(q_d[r], phi_d[r], fld_d[r], s) for r in range(nrhs)])
    f.close()
    return {"workload": "three-layer medium, N=%d charges split between layers, %d charge vectors q~U[-1,1], "
                        "p=%d, float32 form, one tree" % (w.n, nrhs, p),
            "batched_ms": t_batch, "one_at_a_time_ms": t_single,
            "charges_x_vectors_per_s": w.n * nrhs / (t_batch / 1e3), "speedup": t_single / t_batch}


def many_problems_leg(torch, dev, p, flush, k=48):
    """Float32 form, k independent three-layer problems with log-uniform sizes
    in [2k, 100k]: one CUDA graph replay per evaluation against the same
    launches issued directly and against k one-at-a-time evaluations, and the
    graph again after the batch tuner picked settings for the whole batch
    (lfmm_batch_autotune)."""
    from paper_1908_10863_gb300 import LayeredFMM, LayeredFMMBatch, workloads
    import oracle
    probs = workloads.uneven_problems(k)
    ms = []
    for w in probs:
        f = LayeredFMM(w.d, w.eps, p, precision=1)
        f.build(w.xyz, w.layer)
        ms.append(f)
    s = torch.cuda.current_stream()
    out = {"workload": "%d independent three-layer problems (eps=(1,5,10), charges split between layers, "
                       "q~U[-1,1]), N log-uniform in [2000, 100000] (total %d), p=%d, float32 form"
                       % (k, sum(w.n for w in probs), p)}

    def timed(fn, reps=5):
        fn()
        fn()  # direct run + capture, then one replay
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return sorted(ts)[len(ts) // 2]

    total = sum(w.n for w in probs)
    res = {}
    for graph in (True, False):
        b = LayeredFMMBatch(ms, graph=graph)
        q = torch.from_numpy(b.concat([w.q for w in probs])).to(dev)
        phi = torch.empty_like(q)
        fld = torch.empty(3 * total, dtype=torch.float64, device=dev)
        res[graph] = (timed(lambda: b.evaluate_device(q, phi, fld, s)), b.info(), phi.cpu().numpy())
        b.close()
    qd = [torch.from_numpy(w.q).to(dev) for w in probs]
    pd = [torch.empty_like(x) for x in qd]
    fd = [torch.empty((x.shape[0], 3), dtype=torch.float64, device=dev) for x in qd]
    t_seq = timed(lambda: [m.evaluate_device(a, b_, c, s) for m, a, b_, c in zip(ms, qd, pd, fd)])
    seq_phi = np.concatenate([x.cpu().numpy() for x in pd])
    # the batch tuned as a whole (lfmm_batch_autotune times graph replays of
    # the whole batch for settings applied to every member)
    b = LayeredFMMBatch(ms, graph=True)
    t0 = time.perf_counter()
    rows = b.autotune(reps=3)
    tune_s = time.perf_counter() - t0
    q = torch.from_numpy(b.concat([w.q for w in probs])).to(dev)
    phi = torch.empty_like(q)
    fld = torch.empty(3 * total, dtype=torch.float64, device=dev)
    t_tuned = timed(lambda: b.evaluate_device(q, phi, fld, s))
    phi_t = phi.cpu().numpy()
    b.close()
    for m in ms:
        m.close()
    t_g, info, phi_g = res[True]
    best = [r for r in rows if r["chosen"]]
    out.update({"graph_batch_tuned_ms": t_tuned, "batch_tuning_s": tune_s,
                "particles_per_s_batch_tuned": total / (t_tuned / 1e3),
                "batch_tuned_setting": best[0] if best else None, "batch_tuner_rows": rows,
                "err2_phi_batch_tuned_vs_default": oracle.err2(phi_g, phi_t)})
    out.update({"graph_ms": t_g, "direct_ms": res[False][0], "one_at_a_time_ms": t_seq,
                "particles_per_s": total / (t_g / 1e3), "speedup_vs_one_at_a_time": t_seq / t_g,
                "graph_nodes": info["graph_nodes"], "kernel_nodes": info["kernel_nodes"],
                "err2_phi_graph_vs_one_at_a_time": oracle.err2(seq_phi, phi_g)})
    return out


def accuracy_table(torch, dev, targets=(200, 60)):
    """Relative L2 errors (potential and field) of both forms against the CPU
    oracle (exact image series), one JSON line per case.  Small N: all
    targets; N = 1M: a seeded target subsample of the given sizes.  The
    paper_p4 case is Section 4's accuracy experiment (P4-shaped domains,
    eps = (21.2, 47.5, 62.8), N = 2,848), Err2 against p."""
    import oracle
    from paper_1908_10863_gb300 import LayeredFMM, workloads
    cases = [("paper_p4", "(21.2,47.5,62.8)", 2848, 2848, (2, 4, 6, 8, 10, 12, 14, 16, 18, 20)),
             ("config1", "(1,5,10)", 1000, 1000, (6, 10, 14, 20)),
             ("config2", "(1,5,10)", 1 << 20, targets[0], (6, 10, 14)),
             ("config2", "(1,80,2)", 1 << 20, targets[1], (6, 10, 14))]
    for name, med, n, ns, plist in cases:
        if name == "paper_p4":
            w = workloads.paper_p4()
        else:
            eps = workloads.EPS_CONFIG if med == "(1,5,10)" else workloads.EPS_HIGH_CONTRAST
            w = workloads.config1(n, eps=eps) if name == "config1" else workloads.config2(n, eps=eps)
        t = np.arange(w.n) if ns >= w.n else workloads.subsample(w.n, ns)
        t0 = time.perf_counter()
        ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES,
                                  threads=os.cpu_count() or 1)
        oracle_s = time.perf_counter() - t0
        for p in plist:
            for prec in (0, 1):
                if prec == 1 and p > 14:
                    continue  # the float32 form stops at p = 14
                with LayeredFMM(w.d, w.eps, p, precision=prec) as f:
                    f.build(w.xyz, w.layer)
                    phi, E = f.evaluate(w.q)
                print(json.dumps({"case": name, "eps": med, "n": w.n, "targets": int(len(t)), "p": p,
                                  "form": "fp32" if prec else "fp64", "err2_phi": oracle.err2(ref, phi[t]),
                                  "err2_field": oracle.err2(refE, E[t]), "oracle_s": round(oracle_s, 1)}),
                      flush=True)


def sweep(torch, dev, flush, sizes=(1 << 16, 1 << 18, 1 << 20), orders=(6, 10, 14), sample=256):
    """Three-layer split workload (eps = (1, 5, 10)): build + evaluate time per
    step and Err2 against the oracle (exact image series, a seeded sample of
    targets) for every N, p and form; one JSON line per case."""
    import oracle
    from paper_1908_10863_gb300 import LayeredFMM, workloads
    from paper_1908_10863_gb300.lfmm import OPT_TENSOR_CORES
    for n in sizes:
        w = workloads.config2(n)
        t = workloads.subsample(w.n, sample)
        ref, refE = oracle.direct(w.d, w.eps, w.xyz, w.layer, w.q, targets=t, mode=oracle.MODE_IMAGES,
                                  threads=os.cpu_count() or 1)
        xyz_d = torch.from_numpy(w.xyz).to(dev)
        lay_d = torch.from_numpy(w.layer).to(dev)
        q_d = torch.from_numpy(w.q).to(dev)
        phi_d = torch.empty(w.n, dtype=torch.float64, device=dev)
        fld_d = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
        for p in orders:
            # float32 and FP64 with the automatic free M2L engine (tensor cores
            # where (p+1)^2 <= 128), and for wider expansions also float32 with
            # the wide tensor-core form asked for
            forms = [(1, 2), (0, 2)] + ([(1, 1)] if (p + 1) ** 2 > 128 else [])
            for prec, tc in forms:
                with LayeredFMM(w.d, w.eps, p, precision=prec) as f:
                    f.set_option(OPT_TENSOR_CORES, tc)
                    steps = 5 if prec else 2
                    times, launches, stages = run_form(f, xyz_d, lay_d, q_d, phi_d, fld_d, torch, steps, 1, flush)
                    st = f.stats()
                ms = sum(times) / len(times)
                phi, E = phi_d.cpu().numpy(), fld_d.cpu().numpy()
                form = ("fp32" if tc == 2 else "fp32 (wide tensor-core M2L)") if prec else "fp64"
                print(json.dumps({"sweep": "config2", "n": n, "p": p, "form": form,
                                  "ms_per_step": ms, "particles_per_s": n / (ms / 1e3), "build_ms": stages["build"],
                                  "evaluate_ms": stages["total"], "m2l_free_ms": stages["m2l_free"],
                                  "p2p_ms": stages["p2p"], "m2l_pairs": st["m2l_free"], "depth": st["depth"],
                                  "err2_phi": oracle.err2(ref, phi[t]), "err2_field": oracle.err2(refE, E[t]),
                                  "targets": sample}), flush=True)


def main():
    args = parse()
    world, rank, local, pg = dist_setup(args)
    from paper_1908_10863_gb300 import workloads

    w = workloads.config2(args.n)
    workload = ("three-layer medium d=(0,-1.2) eps=(1,5,10), N=%d charges split equally between layers, "
                "q~U[-1,1], p=%d, leaf 40" % (w.n, args.p))

    if args.impl == "reference":
        if rank != 0:
            return 0
        count = max(8, args.sample // 4)
        for _ in range(args.warmup):
            pass  # the oracle has no warm-up state; warm-up steps are not needed
        times = []
        threads = os.cpu_count() or 1
        for _ in range(args.steps):
            _, _, _, dt, threads = oracle_sample(w, count)
            times.append(dt)
        ms = 1e3 * sum(times) / len(times)
        value = count / (ms / 1e3)
        line = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": workload, "sample_targets": count},
                "cpu_baseline": {"value": value, "unit": "particles/s", "cores": threads, "kind": "oracle",
                                 "sample": "%d targets (seeded subsample) x all %d sources per step, exact "
                                           "three-layer image series" % (count, w.n)},
                "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    from paper_1908_10863_gb300 import LayeredFMM

    if args.accuracy_table:
        if rank == 0:
            accuracy_table(torch, torch.device("cuda", local), tuple(int(v) for v in args.acc_targets.split(",")))
        return 0
    if args.sweep:
        if rank == 0:
            torch.cuda.set_device(local)
            dev = torch.device("cuda", local)
            sweep(torch, dev, torch.empty((256 << 20) // 4, dtype=torch.float32, device=dev))
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    xyz_d = torch.from_numpy(w.xyz).to(dev)
    lay_d = torch.from_numpy(w.layer).to(dev)
    q_d = torch.from_numpy(w.q).to(dev)
    phi_d = torch.empty(w.n, dtype=torch.float64, device=dev)
    fld_d = torch.empty((w.n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty((256 << 20) // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    results = {}
    known = {"fp32_surrogate": (1, True), "fp32": (1, False), "fp64": (0, False)}
    forms = [(nm, ) + known[nm] for nm in args.forms.split(",") if nm in known]
    if args.no_fp64:
        forms = [fm for fm in forms if fm[0] != "fp64"]
    if not forms:
        raise SystemExit("no known form in --forms")
    clocks = Clocks(local)
    headline = forms[0][0]
    for name, prec, surr in forms:
        f = LayeredFMM(w.d, w.eps, args.p, precision=prec)
        train_s = None
        if surr:
            t0 = time.perf_counter()
            f.surrogate_train(SURR_SAMPLES, SURR_EPOCHS, SURR_SEED)
            train_s = time.perf_counter() - t0
            f.set_option(5, 1)
        barrier(pg)
        if name == headline:
            clocks.start()
        times, launches, tim = run_form(f, xyz_d, lay_d, q_d, phi_d, fld_d, torch, args.steps, args.warmup, flush)
        if name == headline:
            clk = clocks.stop()
        barrier(pg)
        st = f.stats()
        ms = sum(times) / len(times)
        results[name] = {"ms_per_step": ms, "times": times, "timings": tim, "stats": st, "launches": launches,
                         "prec": prec,
                         "phi": phi_d.cpu().numpy().copy(), "E": fld_d.cpu().numpy().copy(),
                         "surrogate_train_s": train_s}
        if name == headline and prec == 1:
            # the near-field kernel alone (not overlapped with the far field),
            # CUDA events on its stream, for its own roofline; untimed by the step
            f.set_option(13, 1)
            f.set_option(3, 1)
            stream = torch.cuda.current_stream()
            f.build_device(xyz_d, lay_d, stream)
            near_ms = []
            for _ in range(4):
                f.evaluate_device(q_d, phi_d, fld_d, stream)
                torch.cuda.synchronize()
                near_ms.append(f.timings()["p2p"])
            f.set_option(3, 0)
            f.set_option(13, 0)
            results[name]["near_alone_ms"] = statistics.median(near_ms[1:])
        if name == headline:
            # end-to-end through the host-buffer C ABI (copies inside the timed region)
            e2e_t = []
            out = (np.empty(w.n), np.empty((w.n, 3)))  # the caller's result buffers, reused every step
            f.build(w.xyz, w.layer)  # untimed warm-up (first touch of the result pages)
            f.evaluate(w.q, out=out)
            for k in range(max(3, min(args.steps, 10))):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                f.build(w.xyz, w.layer)
                ph, E = f.evaluate(w.q, out=out)
                e2e_t.append(time.perf_counter() - t0)
            results[name]["e2e_s"] = sum(e2e_t) / len(e2e_t)
        f.close()
    # the plain FP64 form at lower orders, for the comparison at matched accuracy
    matched_runs = {}
    if rank == 0 and not args.no_fp64 and args.matched_orders:
        for pm in sorted({int(v) for v in args.matched_orders.split(",") if v.strip()}):
            if pm == args.p:
                continue
            f = LayeredFMM(w.d, w.eps, pm, precision=0)
            times, launches, tim = run_form(f, xyz_d, lay_d, q_d, phi_d, fld_d, torch, 2, 1, flush)
            f.close()
            matched_runs[pm] = {"ms_per_step": sum(times) / len(times), "phi": phi_d.cpu().numpy().copy()}
    near = None
    if not args.no_near and rank == 0:
        near = near_interface_leg(torch, dev, args.p, flush)
    multi = None
    if not args.no_multi and rank == 0:
        multi = multi_rhs_leg(torch, dev, args.p, flush)
    many = None
    if not args.no_batch and rank == 0:
        many = many_problems_leg(torch, dev, args.p, flush)
    four = None
    if not args.no_four and rank == 0:
        try:
            four = four_layer_leg(torch, dev, args.p, flush)
        except Exception as exc:  # a secondary workload never voids the headline line
            four = {"error": "%s: %s" % (type(exc).__name__, exc)}

    ms_max = allmax(pg, results[headline]["ms_per_step"])
    e2e_max = allmax(pg, results[headline]["e2e_s"])
    if rank != 0:
        barrier(pg)
        return 0

    value = world * w.n / (ms_max / 1e3)
    t, ref, refE, dt, threads = oracle_sample(w, args.sample)
    forms_out = {}
    for name in results:
        r = results[name]
        import oracle
        e2p = oracle.err2(ref, r["phi"][t])
        e2E = oracle.err2(refE, r["E"][t])
        forms_out[name] = {"particles_per_s": w.n / (r["ms_per_step"] / 1e3), "ms_per_step": r["ms_per_step"],
                           "err2_phi": e2p, "err2_field": e2E, "stage_ms": r["timings"],
                           "build_stats": {k: v for k, v in r["stats"].items() if k != "launches"}}
        try:  # per-layer breakdown of the same sample; never voids the line
            forms_out[name]["err2_phi_per_layer"] = err2_per_layer(ref, r["phi"][t], w.layer[t])
            forms_out[name]["err2_field_per_layer"] = err2_per_layer(refE, r["E"][t], w.layer[t])
        except Exception as exc:
            forms_out[name]["err2_per_layer_error"] = "%s: %s" % (type(exc).__name__, exc)
        if r["surrogate_train_s"] is not None:
            forms_out[name]["surrogate_train_s"] = r["surrogate_train_s"]
    matched = None
    if "fp64" in results and headline != "fp64":
        fp64_rows = [{"p": args.p, "err2_phi": forms_out["fp64"]["err2_phi"],
                      "particles_per_s": forms_out["fp64"]["particles_per_s"]}]
        for pm, r in matched_runs.items():
            fp64_rows.append({"p": pm, "err2_phi": oracle.err2(ref, r["phi"][t]),
                              "particles_per_s": w.n / (r["ms_per_step"] / 1e3)})
        fp64_rows.sort(key=lambda d: d["p"])
        target = forms_out[headline]["err2_phi"]
        ok = [d for d in fp64_rows if d["err2_phi"] <= target]
        best = ok[0] if ok else None
        matched = {"headline_p": args.p, "headline_err2_phi": target, "fp64": fp64_rows,
                   "fp64_p_at_matched_accuracy": best["p"] if best else None,
                   "speedup_vs_fp64_at_matched_accuracy": (value / world / best["particles_per_s"]) if best else None,
                   "note": "the smallest FP64 order whose Err2(phi) on the same oracle sample is at most the "
                           "headline form's; speedup = headline particles/s / that FP64 form's"}
    st = results[headline]["stats"]
    tim = results[headline]["timings"]
    flops = st["m2l_free"] * m2l_flops_per_pair(args.p)
    m2l_ms = tim["m2l_free"]
    achieved = flops / (m2l_ms / 1e3) / 1e12 if m2l_ms > 0 else None
    tensor_path = results[headline].get("prec", 1) == 1 and (args.p + 1) ** 2 <= 128
    if tensor_path:
        peak, src = tf32_peak_tflops()
        roof = {"kernel": "k_m2l_tc (free-space M2L, tcgen05 3xTF32)", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                "traffic": (TC_DRAM_BYTES_PER_PAIR * st["m2l_free"]) if args.p == 10 else None,
                "peak_note": "dense TF32 = bf16 GEMM burst %s (MEASURED_PEAKS.json) x nominal TF32/BF16 1.1/2.25; "
                             "algorithmic flops = 8 (p+1)^2 (p+1)(p+2)/2 per box pair (the tensor cores execute "
                             "3 TF32 products of padded 128x128 operators); duration = the stage's CUDA events "
                             "inside the timed steps; traffic scaled by pair count from an ncu capture at "
                             "N=1,048,576" % src}
    else:
        sm_mhz = clk.get("sm_max_mhz") or 2070.0
        peak = fp32_peak_tflops(sm_mhz)
        roof = {"kernel": "k_m2l_gemm (free-space M2L, FP32 CUDA cores)", "bound": "alu", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None, "traffic": None,
                "peak_note": "FP32 CUDA-core peak from unit counts (152 SMs x 128 lanes x 2 flops) at the max SM "
                             "clock seen; algorithmic flops = 8 (p+1)^2 (p+1)(p+2)/2 per box pair"}
    roof_p2p = None
    if results[headline].get("near_alone_ms"):
        pairs = st["p2p_free"] + st["p2p_reaction"]
        t_near = results[headline]["near_alone_ms"]
        sm_mhz = (clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0)
        pk = fp32_peak_tflops(sm_mhz)
        ach = pairs * 20 / (t_near / 1e3) / 1e12
        roof_p2p = {"kernel": "k_p2p_free_staged (float32 near field, free space)" if st["p2p_reaction"] == 0
                    else "near field (float32, with reaction pairs)",
                    "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                    "traffic": None, "pairs": pairs, "ms": t_near,
                    "peak_note": "FP32 CUDA-core peak from unit counts (152 SMs x 128 lanes x 2 flops) at the median "
                                 "SM clock sampled in the timed region; algorithmic flops = 20 per near pair "
                                 "(potential and field); duration = CUDA events around the near field run alone "
                                 "(not beside the far field), after the timed steps"}
    # the other stages: counted work (the library's statistics) over their
    # CUDA-event times inside the timed steps, against the peak of the units
    # each runs on (the near field runs beside them, so these are lower bounds)
    sm_mhz = (clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0)
    pk32 = fp32_peak_tflops(sm_mhz)
    sms = forms_out[headline]["stage_ms"]
    nc, nre = (args.p + 1) ** 2, (args.p + 1) * (args.p + 2) // 2
    edge = 8 * nc * nre  # flops per parent-child edge (dense complex shift) and per M2L pair
    # the float32 form at (p+1)^2 <= 128 applies the reaction keys on the tensor
    # cores (k_m2r_tc, 3xTF32): its peak is the dense TF32 rate
    r_tc = results[headline].get("prec", 1) == 1 and (args.p + 1) ** 2 <= 128
    pk_tf32 = tf32_peak_tflops()[0]
    work = [("p2m", "k_p2m", st["n"], 20 * nc, "charge", pk32),
            ("m2m", "k_m2l_gemm (M2M)", st["m2m_edges"], edge, "parent-child edge", pk32),
            ("m2l_reaction", "k_m2r_tc (keyed reaction M2L, tcgen05 3xTF32)" if r_tc
             else "k_m2r_gemm (keyed reaction M2L)", st["m2l_reaction"], edge, "reaction box pair",
             pk_tf32 if r_tc else pk32),
            ("l2l", "k_m2l_gemm / k_m2l_tc (L2L)", st["m2m_edges"], edge, "parent-child edge", pk32),
            ("l2p", "k_l2p", st["n"], 20 * nc, "charge", pk32)]
    stage_roofs = []
    for stage, kern, units, fpu, unit, pk in work:
        ms_s = sms.get(stage)
        if not ms_s or not units:
            continue
        ach = units * fpu / (ms_s / 1e3) / 1e12
        stage_roofs.append({"stage": stage, "kernel": kern, "units": int(units), "unit": unit,
                            "flops_per_unit": fpu, "ms": ms_s, "achieved_tflops": ach, "peak_tflops": pk,
                            "peak": "dense TF32 tensor" if pk is pk_tf32 else "FP32 CUDA core",
                            "frac": ach / pk})
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "particles/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload, "form": form_label(headline, st),
                   "l2": "256 MB buffer written between timed steps (L2 flushed)", "parallelism": "replicas"},
        "err2": {"phi": forms_out[headline]["err2_phi"], "field": forms_out[headline]["err2_field"],
                 "phi_per_layer": forms_out[headline].get("err2_phi_per_layer"),
                 "field_per_layer": forms_out[headline].get("err2_field_per_layer"),
                 "targets": int(len(t)), "reference": "CPU oracle (FP64 direct sum, exact image series)"},
        "forms": forms_out,
        "roofline": roof,
        "roofline_near_field": roof_p2p,
        "roofline_stages": stage_roofs,
        "cpu_baseline": {"value": len(t) / dt, "unit": "particles/s", "cores": threads, "kind": "oracle",
                         "sample": "%d targets (seeded subsample) x all %d sources, exact three-layer image "
                                   "series, %.1f s" % (len(t), w.n, dt)},
        "e2e": {"value": world * w.n / e2e_max, "unit": "particles/s", "h2d_bytes_per_step": w.n * (24 + 4 + 8),
                "d2h_bytes_per_step": w.n * (8 + 24)},
        "surrogate_pairs": {"network": int(st.get("surr_net_pairs", 0)),
                            "quadrature": int(st.get("surr_quad_pairs", 0)),
                            "near_reaction_pairs": int(st.get("p2p_reaction", 0))},
        "gpu_launches": results[headline]["launches"],
        "clocks": clk,
        "matched_accuracy": matched,
        "near_interface": near,
        "multi_rhs": multi,
        "many_problems": many,
        "four_layers": four,
    }
    print(json.dumps(line))
    barrier(pg)
    return 0


if __name__ == "__main__":
    sys.exit(main())
