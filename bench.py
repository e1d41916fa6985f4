#!/usr/bin/env python3
"""Throughput of the factorized stochastic three-point hot path on one GB300.

One step = one pass of the whole hot path over the meson workload on a 24^3 x 48
lattice: for each sink separation t_f in {8, 10, 12} (source at the origin, its
own 16 Z2xZ2 noises and Gaussian solutions), the insertion part on every slice
0..t_f, the meson spectator on t_f (93 momenta with |k|^2 <= 8 at sink and
insertion), and the combine for 16 Gamma structures on every insertion slice.

Metric: site*noise*momentum contractions per second = sum over projected slices
of V3 * N_r * Nq, divided by the wall time of the step (timed on the device).

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
      python bench.py --impl reference      (the FP64 CPU oracle on a bounded sample)
"""
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

METRIC = "site*noise*mom contractions/s"
UNIT = "contractions/s"
WORKLOAD = "meson 3pt 24^3x48, 1 source at origin, N_r=16, t_f in {8,10,12}, 93 momenta (|k|^2<=8), complex128 inputs"

L, T_SLAB, N_R, TFS, N2MAX = 24, 13, 16, (8, 10, 12), 8
SEED = 2000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lhc", choices=["lhc", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="leave out the plain FP64 GPU comparator")
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the FP64 comparator")
    ap.add_argument("--serve-jobs", type=int, default=100,
                    help="jobs of the served stream reported beside the headline (0 leaves it out)")
    ap.add_argument("--streams", type=int, default=3,
                    help="contexts and streams the step's three t_f sets are spread over (their kernels overlap)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the heuristic launch shapes instead of autotuning them during warm-up")
    ap.add_argument("--workload", default="meson24",
                    choices=["meson24", "baryon32", "batched", "serve", "mom1", "allmom", "paper", "extras",
                             "smallcalls"],
                    help="meson24: the headline line; the others measure the further benchmark rows")
    return ap.parse_args()


def units_per_step(nq):
    V3 = L ** 3
    slices = sum(tf + 1 for tf in TFS) + len(TFS)
    return V3 * N_R * nq * slices


# --------------------------------------------------------------------------- inputs

def make_inputs():
    """Seeded inputs of the workload (host, numpy): S on slices 0..12 (the slab the
    step touches), and per t_f its own solutions (slices 0..t_f) and noise."""
    from paper_1711_02384_gb300 import inputs
    S = inputs.propagator(SEED, L, 48, slices=range(T_SLAB))              # [13][V3][12][12]
    psis, etas = [], []
    for j, tf in enumerate(TFS):
        psi = np.zeros((N_R, T_SLAB, L ** 3, 12), dtype=np.complex128)
        psi[:, :tf + 1] = inputs.solutions(SEED + 10 * (j + 1), L, 48, N_R, slices=range(tf + 1))
        psis.append(psi)
        etas.append(inputs.noise(SEED + 10 * (j + 1) + 3, L, N_R, tf))
    return S, psis, etas


def gamma_sets():
    """Gamma_snk, Gamma_ins, Gamma_src of the combine: the 16 Dirac structures at sink and
    source, gamma_4 at the insertion."""
    from paper_1711_02384_gb300 import inputs
    g16 = inputs.dirac_structures()
    g4 = np.broadcast_to(inputs.dirac_matrices()[3], (16, 4, 4)).copy()
    return g16, g4, g16.copy()


# --------------------------------------------------------------------------- clocks

def nvsmi_id(local):
    """The id under which nvidia-smi knows CUDA device `local`: its PCI bus id (or, where
    torch does not report one, its UUID).  nvidia-smi ignores CUDA_VISIBLE_DEVICES, so the
    CUDA ordinal can name another GPU of the machine than the one being timed."""
    import torch
    p = torch.cuda.get_device_properties(local)
    bus, slot = getattr(p, "pci_bus_id", None), getattr(p, "pci_device_id", None)
    if bus is not None and slot is not None:
        return f"{int(getattr(p, 'pci_domain_id', 0) or 0):08X}:{int(bus):02X}:{int(slot):02X}.0"
    u = getattr(p, "uuid", None)
    if u is not None:
        u = str(u)
        return u if u.startswith("GPU-") else "GPU-" + u
    return str(local)


def link_rates(dev, stream, mib=512, reps=3, trials=3):
    """This box's pinned-copy rates in each direction, GB/s: the best of `trials` timings
    (CUDA events on `stream`) of `reps` copies of a `mib` MiB buffer."""
    import torch
    h = torch.empty(mib << 20, dtype=torch.uint8).pin_memory()
    d = torch.empty(mib << 20, dtype=torch.uint8, device=dev)
    rate = {}
    for name, dst, src in (("h2d_gbs", d, h), ("d2h_gbs", h, d)):
        best = 0.0
        with torch.cuda.stream(stream):
            dst.copy_(src, non_blocking=True)
            for _ in range(trials):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    dst.copy_(src, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                best = max(best, reps * (mib << 20) / (e0.elapsed_time(e1) * 1e6))
        rate[name] = best
    return rate


def host_link(before, after, h2d_bytes, d2h_bytes, ms_per_step):
    """The host link around the end-to-end steps: the rates measured before and after them,
    the floor that the better of the two puts on one step's copies (both directions
    overlap, so the slower direction), and the fraction of that floor reached."""
    h2d = max(before["h2d_gbs"], after["h2d_gbs"])
    d2h = max(before["d2h_gbs"], after["d2h_gbs"])
    floor = max(h2d_bytes / h2d, d2h_bytes / d2h) / 1e6
    return {"before": before, "after": after, "floor_ms": floor, "frac_of_floor": floor / ms_per_step}


class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 25

    def __init__(self, gpu_id, window="timed steps"):
        """gpu_id: nvidia-smi's id of the timed GPU (nvsmi_id)."""
        self.idx = gpu_id
        self.window = window
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self, ready_s=2.0):
        """Starts sampling every INTERVAL_MS and waits (at most ready_s) for the first
        sample, so that the steps that follow are covered from their start."""
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < ready_s and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "gpu_id": self.idx}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "window": self.window,
                "interval_ms": self.INTERVAL_MS, "gpu_id": self.idx}


# --------------------------------------------------------------------------- replicas

def max_over_ranks(x, world, device="cpu"):
    """The largest x over the ranks of the job: the slowest replica's time is the job's."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step, steps, world, ms):
    """Whole-job throughput: the units every replica processed over the slowest one's time."""
    return units_per_step * steps * world / (ms / 1e3)


# --------------------------------------------------------------------------- reference arm / cpu baseline

SAMPLE = ("insertion slice 5 + spectator slice 10 of the t_f=10 set (16 noises, 93 momenta) and the "
          "combine of that slice for the 16 Gamma structures")


def oracle_sample(S, psis, etas, k):
    """The FP64 oracle as it stands on a bounded sample of the workload: the insertion
    on slice 5 and the spectator on the sink slice, for t_f = 10 (all 16 noises, all 93
    momenta), and the combine of that slice for the step's 16 Gamma structures.
    Returns (units, seconds, (insertion, spectator, correlators))."""
    from oracle import contractions as OC
    g5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(complex)
    r3 = np.zeros(3, dtype=int)
    g_snk, g_ins, g_src = gamma_sets()
    t0 = time.perf_counter()
    ins = OC.insertion(S[5:6], psis[1][:, 5:6], g5, r3, k, L)
    spec = OC.spectator_meson(S[TFS[1]], etas[1], g5, r3, k, L)
    corr = OC.combine_meson(spec, ins[0], g_snk, g_ins, g_src)
    dt = time.perf_counter() - t0
    return 2 * L ** 3 * N_R * len(k), dt, (ins[0], spec, corr)


def parity_errors(ins, spec, corr, ref):
    """Errors of the GPU outputs of the sampled slices against the oracle's, per
    correlator: for the insertion and spectator parts the largest normwise error of a
    block (one momentum over all open components and noises); for the combine the
    largest |C_gpu - C_ref| of a correlator over the largest |C_ref| of its row (the same
    Gamma structure and sink momentum, all insertion momenta)."""
    ri, rs, rc = ref

    def blocks(got, want):
        got, want = got.reshape(want.shape[0], -1), want.reshape(want.shape[0], -1)
        return float(np.max(np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)))

    row = np.max(np.abs(rc), axis=-1, keepdims=True)
    return {"insertion": blocks(ins, ri), "spectator": blocks(spec, rs),
            "combine": float(np.max(np.abs(corr - rc) / row))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.momenta import momenta
    k = momenta(N2MAX)
    S, psis, etas = make_inputs()
    for _ in range(args.warmup):
        oracle_sample(S, psis, etas, k)
    tot_u, tot_t = 0, 0.0
    for _ in range(args.steps):
        u, t, _ = oracle_sample(S, psis, etas, k)
        tot_u += u
        tot_t += t
    v = tot_u / tot_t
    cores = os.cpu_count()
    sample = SAMPLE + ", per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Philox Gaussian propagators/solutions, Z2xZ2 noise)",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload != "meson24":
        import bench_workloads
        bench_workloads.run(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1711_02384_gb300 import lhc
    k = lhc.momenta(N2MAX)
    nq = len(k)
    r = np.zeros(4, dtype=np.int32)
    S_h, psis_h, etas_h = make_inputs()
    g16, g4, gsrc = gamma_sets()
    S = torch.from_numpy(S_h).to(dev)
    psis = [torch.from_numpy(p).to(dev) for p in psis_h]
    etas = [torch.from_numpy(e).to(dev) for e in etas_h]
    G = [torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (g16, g4, gsrc)]
    ctx = lhc.Context(local)
    ctx.set_tuning(not args.no_tune)   # new shapes are tuned in the first warm-up step
    st = torch.cuda.current_stream(dev)

    outs_ins = [torch.empty((tf + 1, nq, N_R, 192), dtype=torch.complex128, device=dev) for tf in TFS]
    outs_spec = [torch.empty((nq, N_R, 192), dtype=torch.complex128, device=dev) for _ in TFS]
    outs_c = [torch.empty((tf + 1, 16, nq, nq), dtype=torch.complex128, device=dev) for tf in TFS]

    # the three t_f sets are independent chains (insertion -> spectator -> combine); with
    # --streams n they go to n contexts on n streams, so one set's memory-bound kernels
    # overlap another's fused kernel
    nstr = max(1, min(args.streams, len(TFS)))
    ctxs = [ctx] + [lhc.Context(local) for _ in range(nstr - 1)]
    sts = [st] + [torch.cuda.Stream(dev) for _ in range(nstr - 1)]

    def step_on(cs, ss):
        # the propagator slices 0..12 are narrowed once per step and shared by the six
        # calls (the FP64 comparator reads complex128 directly)
        if args.prec == "mixed":
            cs[0].stage_propagator(S, 0, T_SLAB - 1, stream=ss[0].cuda_stream)
        for s in ss[1:]:
            s.wait_stream(ss[0])
        for j, tf in enumerate(TFS):
            c, s = cs[j % len(cs)], ss[j % len(ss)].cuda_stream
            c.insertion(S, psis[j], 0, tf, r, k, prec=args.prec, out=outs_ins[j], stream=s)
            c.spectator(S, etas[j], tf, r, k, prec=args.prec, out=outs_spec[j], stream=s)
            c.combine(outs_spec[j], outs_ins[j], G[0], G[1], G[2], prec=args.prec, out=outs_c[j], stream=s)
        for s in ss[1:]:
            ss[0].wait_stream(s)

    def step():
        step_on(ctxs, sts)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # launch shapes are tuned on one stream first: candidates timed next to other work
    # would be picked for the wrong conditions
    step_on([ctx], [st])
    # clocks are sampled every 25 ms from the warm-up through the end-to-end steps: the
    # timed region alone (20 steps, about 60 ms) would hold only a few samples
    clocks = Clocks(nvsmi_id(local), window="warm-up, timed and end-to-end steps of the mixed path")
    clocks.start()
    for _ in range(args.warmup):
        step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_launch0 = lhc.launch_count()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    barrier()
    for c in ctxs:   # a kernel that gave up a bounded wait raises here instead of giving a number
        c.sync()
    n_launches = lhc.launch_count() - n_launch0
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world, dev)
    upstep = units_per_step(nq)
    value = job_value(upstep, args.steps, world, ms)

    # dominant kernel: timed with CUDA events on its own stream by the library
    kern = lhc.KERNEL_FUSED if args.prec == "mixed" else lhc.KERNEL_PROJECT
    # (one context on one stream: every kernel of the step is timed alone)
    ctx.profile(True)
    step_on([ctx], [st])
    torch.cuda.synchronize(dev)
    ctx.profile(False)
    kms, kn, kwork = ctx.profile_read(kern)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    if args.prec == "mixed":
        peak = peaks.get("bf16_tflops", 1900.0)
        bound, punit, peak_src = "tensor", "TFLOP/s", "measured bf16 burst (fp16 same rate)"
    else:
        peak = 1.25     # FP64: 2 DFMA/clk/SM x 152 SMs x ~2.06 GHz (nominal GB300 FP64 rate)
        bound, punit, peak_src = "alu", "TFLOP/s", "nominal FP64 1.25 TFLOP/s"
    achieved = (kwork / (kms / 1e3)) / 1e12 if kms > 0 else None
    # DRAM bytes per launch: ncu dram__bytes_read + dram__bytes_write of the same kernel on
    # the 2-slice 24^3 case (83.07 MB for 4.11e7 units: 2.02 bytes per unit, the compulsory
    # input), scaled to this workload's units per launch
    traffic = 2.02 * upstep / kn if (args.prec == "mixed" and kn) else None
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": punit,
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "kernel_ms_per_launch": kms / kn if kn else None, "launches_per_step": kn,
                "peak_source": peak_src}
    kernels = {}
    for kid, name in enumerate(lhc.KERNEL_NAMES):
        kms_i, kn_i, _ = ctx.profile_read(kid)
        if kn_i:
            kernels[name] = {"ms_per_step": kms_i, "launches_per_step": kn_i}
    # the sampled slices' outputs of the path timed above, for the parity check against the
    # oracle (the end-to-end leg below reuses the output buffers)
    got = {args.prec: (outs_ins[1][5].cpu().numpy(), outs_spec[1].cpu().numpy(), outs_c[1][5].cpu().numpy())}

    # End to end, inputs on the host: every step uploads the propagator slices 0..12 once
    # (a plain device copy on a copy stream: the six calls of the step share them), passes
    # the solutions and noise vectors to the library as pinned host buffers (it stages
    # them in call order, overlapping the copies with the kernels of earlier calls), keeps
    # the open-spin outputs on the device for the combine, and reads back to the host both
    # the open-spin outputs (the method's data product) and the correlators (the combine
    # writes them to host memory).  The device copy of the propagator and the open-spin
    # outputs alternate between two buffers by step parity, so a step waits only for the
    # step two back and consecutive steps overlap: the host link stays busy across step
    # boundaries.
    e2e = None
    if not args.no_e2e and rank == 0:
        nS = max(TFS) + 1
        S_p = torch.from_numpy(np.ascontiguousarray(S_h[:nS])).pin_memory()
        S_d = [torch.empty(S_p.shape, dtype=S_p.dtype, device=dev) for _ in range(2)]
        psis_p = [torch.from_numpy(p).pin_memory() for p in psis_h]
        etas_p = [torch.from_numpy(e).pin_memory() for e in etas_h]
        G_p = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (g16, g4, gsrc)]
        G_d = [[torch.empty(g.shape, dtype=g.dtype, device=dev) for g in G_p] for _ in range(2)]
        oi = [outs_ins, [torch.empty_like(o) for o in outs_ins]]
        osp = [outs_spec, [torch.empty_like(o) for o in outs_spec]]
        hi = [torch.empty((tf + 1, nq, N_R, 192), dtype=torch.complex128).pin_memory() for tf in TFS]
        hs = [torch.empty((nq, N_R, 192), dtype=torch.complex128).pin_memory() for _ in TFS]
        hc = [torch.empty((tf + 1, 16, nq, nq), dtype=torch.complex128).pin_memory() for tf in TFS]
        side, up = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        st_done = [torch.cuda.Event(), torch.cuda.Event()]     # kernels of the step done with buffers b
        side_done = [torch.cuda.Event(), torch.cuda.Event()]   # read-backs of the step done with buffers b
        nstep = [0]

        def step_host():
            b = nstep[0] & 1
            nstep[0] += 1
            up.wait_event(st_done[b])           # the step two back has finished with S_d[b], G_d[b]
            with torch.cuda.stream(up):
                S_d[b].copy_(S_p, non_blocking=True)
                for gd, gp in zip(G_d[b], G_p):
                    gd.copy_(gp, non_blocking=True)
            st.wait_stream(up)
            st.wait_event(side_done[b])         # and its read-backs with the open-spin outputs b
            if args.prec == "mixed":            # narrowed once, shared by the six calls
                ctx.stage_propagator(S_d[b], 0, nS - 1, stream=st.cuda_stream)
            for j, tf in enumerate(TFS):
                ctx.insertion(S_d[b], psis_p[j], 0, tf, r, k, prec=args.prec, out=oi[b][j], stream=st.cuda_stream)
                ctx.spectator(S_d[b], etas_p[j], tf, r, k, prec=args.prec, out=osp[b][j], stream=st.cuda_stream)
                ctx.combine(osp[b][j], oi[b][j], G_d[b][0], G_d[b][1], G_d[b][2], prec=args.prec, out=hc[j],
                            stream=st.cuda_stream)
                side.wait_stream(st)          # the open-spin outputs go back while the next set runs
                with torch.cuda.stream(side):
                    hi[j].copy_(oi[b][j], non_blocking=True)
                    hs[j].copy_(osp[b][j], non_blocking=True)
            st_done[b].record(st)
            side_done[b].record(side)

        link_before = link_rates(dev, side)
        for _ in range(max(3, args.warmup)):  # both buffer parities; staging slots sized
            step_host()
        torch.cuda.synchronize(dev)
        ne = max(1, min(args.steps, 10))
        t0 = time.perf_counter()
        issue = 0.0   # host time spent issuing the steps (near dt: the host, not the GPU, bounds them)
        for _ in range(ne):
            ti = time.perf_counter()
            step_host()
            issue += time.perf_counter() - ti
        torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t0) / ne
        ctx.sync()
        V3 = L ** 3
        h2d = S_p.numel() * 16 + sum(g.numel() * 16 for g in G_p)                 # propagator slices, Gammas
        h2d += sum(N_R * (tf + 1) * V3 * 12 * 16 + N_R * V3 * 12 * 16 for tf in TFS)   # psi slices, eta
        d2h = sum(((tf + 1) * nq * N_R * 192 + nq * N_R * 192) * 16 for tf in TFS)     # open-spin outputs
        d2h += sum((tf + 1) * 16 * nq * nq * 16 for tf in TFS)                       # correlators
        link = host_link(link_before, link_rates(dev, side), h2d, d2h, dt * 1e3)
        e2e = {"value": upstep / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": dt * 1e3, "host_issue_ms_per_step": issue / ne * 1e3,
               "pattern": "propagator slices uploaded once per step (double-buffered, steps overlap); "
                          "solutions and noise as pinned host "
                          "buffers through the library; open-spin outputs and correlators read back",
               "link": link}

    clk = clocks.stop()

    # The plain FP64 GPU path on the same workload, one context on one stream (a step
    # takes about a second): the comparator the mixed path is measured against.
    fp64 = None
    if args.prec == "mixed" and not args.no_fp64 and rank == 0:
        def step64():
            for j, tf in enumerate(TFS):
                ctx.insertion(S, psis[j], 0, tf, r, k, prec="fp64", out=outs_ins[j], stream=st.cuda_stream)
                ctx.spectator(S, etas[j], tf, r, k, prec="fp64", out=outs_spec[j], stream=st.cuda_stream)
                ctx.combine(outs_spec[j], outs_ins[j], G[0], G[1], G[2], prec="fp64", out=outs_c[j],
                            stream=st.cuda_stream)
        step64()
        torch.cuda.synchronize(dev)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(st)
        for _ in range(args.fp64_steps):
            step64()
        f1.record(st)
        torch.cuda.synchronize(dev)
        ctx.sync()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        fp64 = {"value": upstep / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": args.fp64_steps,
                "warmup": 1, "ratio_mixed_over_fp64": value / (upstep / (ms64 / 1e3)),
                "path": "plain FP64 GPU path (FP64 contraction, FP64 projection, FP64 combine), one stream"}
        got["fp64"] = (outs_ins[1][5].cpu().numpy(), outs_spec[1].cpu().numpy(), outs_c[1][5].cpu().numpy())

    # A served stream of three-point jobs through the job server (resident propagators,
    # continuous batching): latency percentiles beside the served throughput.
    serve = None
    if args.serve_jobs > 0 and rank == 0:
        import bench_workloads
        gen = torch.Generator(device=dev)
        gen.manual_seed(5001)
        serve = bench_workloads.serve_stream(dev, gen, "mixed", njobs=args.serve_jobs)
        serve["config"] = (f"{args.serve_jobs} Poisson-arriving meson 3pt jobs on resident complex64 propagators "
                           "of 16^3x32, 24^3x48, 32^3x64, 48^3x96, N_r in {8,16,32}, |k|^2<=4..16, "
                           "4 slots, 150 GB budget, arrivals at 0.7 x measured capacity")

    # cpu_baseline: the FP64 oracle as it stands, timed on a bounded sample of the
    # workload; its outputs are also the reference of the parity check of that sample.
    cpu = None
    parity = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        from oracle.momenta import momenta
        u, t, ref = oracle_sample(S_h, psis_h, etas_h, momenta(N2MAX))
        cpu = {"value": u / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": SAMPLE}
        parity = {p: parity_errors(*g, ref) for p, g in got.items()}
        parity["sample"] = SAMPLE
        parity["tolerance"] = {"mixed": 1e-6, "fp64": 1e-12}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f16x2->f32 (mixed)" if args.prec == "mixed" else "f64",
            "data": "synthetic (seeded Philox Gaussian propagators/solutions, Z2xZ2 noise)",
            "config": {"workload": WORKLOAD, "precision": args.prec, "parallelism": f"replicas x{world}",
                       "streams": nstr,
                       "l2": "inputs (2.1 GB per step) larger than L2", "units_per_step": upstep,
                       "launch_shapes": "heuristic" if args.no_tune or args.prec != "mixed" else
                       "autotuned in warm-up: " + "; ".join(
                           f"part {r[0]} nt {r[4]}: NH {r[6]} x {r[5]} reps, {r[7]} splits"
                           for r in lhc.tuning_table() if r[2] == L ** 3 and r[3] == N_R)},
            "clocks": clk, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": n_launches, "kernels": kernels, "fp64_gpu": fp64, "parity": parity,
            "serve": serve,
        }))
    for c in ctxs:
        c.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
