"""Further benchmark rows of the factorized three-point path (driven by bench.py --workload).

baryon32  baryon 3pt on 32^3 x 64: eps-eps spectator of two complex64 propagators (32
          noises, 4 sink separations, 123 momenta with |k|^2 <= 9), insertion on every slice
          up to the sink, baryon combine; mixed precision (or --prec fp64)
batched   16 source positions x 3 sink separations, 16 noises, meson and baryon parts, each
          job with its own momentum set (|k|^2 <= 4 .. 16, 33 to 257 momenta); every call of a
          step captured in one CUDA graph and replayed
serve     a Poisson stream of three-point jobs on 16^3x32 .. 48^3x96 lattices through the job
          server (resident propagators, 150 GB budget): latency p50/p99 and throughput, beside
          the plain FP64 path one job at a time
mom1      the meson 24^3x48 step at 1 momentum vs 93 momenta (the paper's observation that
          many more momenta cost little extra)
allmom    every momentum of a 16^3 slice (4096): the projection as a discrete Fourier
          transform (FP64, and FP32 in the mixed path) against the direct FP64 and mixed
          projections
paper     the paper's own measurement on its lattice shape: 32^3 x 96, source at t = 30,
          sinks 10 slices before and after it, 50 noises on both sink slices, 93 momenta at
          sink and insertion, meson and baryon spectators, one insertion call over both
          directions, combines; time per configuration (the paper quotes about 575 s on 8
          KNL nodes for its whole measurement, as context)
extras    the open-spin combine's 16 x 16 Dirac sweep, the baryon open combine (source spins
          open) and the free-field solver, timed
smallcalls  many small calls (48 sources on 16^3 x 32, 4 noises, uneven momentum sets): the
          persistent batch against the same calls one by one, both from CUDA graphs

Inputs are seeded random device tensors (torch): these rows measure throughput; parity
is the tests' job.  Each row prints one JSON line.
"""
import json
import os
import time

import numpy as np
import torch

import bench as B
from paper_1711_02384_gb300 import lhc

UNIT = "contractions/s"


def _peak():
    p = os.path.join(B.ROOT, "MEASURED_PEAKS.json")
    return json.load(open(p)).get("bf16_tflops", 1900.0) if os.path.exists(p) else 1900.0


def _roofline(ctx):
    kms, kn, kwork = ctx.profile_read(lhc.KERNEL_FUSED)
    ach = kwork / (kms / 1e3) / 1e12 if kms > 0 else None
    peak = _peak()
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": ach / peak if ach else None, "traffic": None,
            "kernel_ms_per_launch": kms / kn if kn else None, "launches_per_step": kn,
            "peak_source": "measured bf16 burst (fp16 same rate)"}


def _timed(step, steps, warmup, dev, stream=None, ctx=None):
    """CUDA-event time of `steps` calls of `step` after `warmup` untimed ones.  With `ctx`,
    the library's error check follows the timed region: a kernel that gave up a bounded
    wait (its results invalid, its time meaningless) raises instead of giving a number."""
    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = B.Clocks(B.nvsmi_id(dev.index))
    clocks.start()
    st = stream or torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = lhc.launch_count()
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    if ctx is not None:
        ctx.sync()
    return e0.elapsed_time(e1), clocks.stop(), lhc.launch_count() - n0


def _rand(shape, dtype, dev, g):
    return torch.randn(shape, dtype=dtype, device=dev, generator=g)


def _line(args, metric, value, ms, workload, extra):
    d = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
         "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
         "dtype": "f32+f16x2->f32 (mixed)" if args.prec == "mixed" else "f64",
         "data": "synthetic (seeded random device tensors)", "config": {"workload": workload, "precision": args.prec,
                    "l2": "inputs of every step larger than L2 (129 MB)"}}
    d.update(extra)
    print(json.dumps(d))


# --------------------------------------------------------------------------- baryon32

def run_baryon32(args, dev, g):
    L, TFS, NR = 32, (8, 10, 12, 14), 32
    V3 = L ** 3
    k = lhc.momenta(9, 3)
    nq = len(k)
    slab = max(TFS) + 1
    GA = _rand((slab, V3, 12, 12), torch.complex64, dev, g)
    GB = _rand((slab, V3, 12, 12), torch.complex64, dev, g)
    psis = [_rand((NR, slab, V3, 12), torch.complex64, dev, g) for _ in TFS]
    etas = [_rand((NR, V3, 12), torch.complex64, dev, g) for _ in TFS]
    ng = 4
    Ws = _rand((ng, 4, 4, 4), torch.complex128, dev, g)
    Gi = _rand((ng, 4, 4), torch.complex128, dev, g)
    Wc = _rand((ng, 4, 4, 4), torch.complex128, dev, g)
    ctx = lhc.Context(0)
    ctx.set_tuning(not args.no_tune)   # new shapes are tuned in the first warm-up step
    r = (0, 0, 0, 0)
    oi = [torch.empty((tf + 1, nq, NR, 192), dtype=torch.complex128, device=dev) for tf in TFS]
    osb = [torch.empty((nq, NR, 3072), dtype=torch.complex128, device=dev) for _ in TFS]
    oc = [torch.empty((tf + 1, ng, nq, nq), dtype=torch.complex128, device=dev) for tf in TFS]

    def step():
        for j, tf in enumerate(TFS):
            ctx.insertion(GA, psis[j], 0, tf, r, k, prec=args.prec, out=oi[j])
            ctx.spectator(GA, etas[j], tf, r, k, prec=args.prec, GB=GB, out=osb[j])
            ctx.combine(osb[j], oi[j], Ws, Gi, Wc, prec=args.prec, out=oc[j])

    ms, clk, nl = _timed(step, args.steps, args.warmup, dev, ctx=ctx)
    units = sum(tf + 2 for tf in TFS) * V3 * NR * nq
    ctx.profile(True)
    step()
    torch.cuda.synchronize(dev)
    ctx.profile(False)
    kern = {}
    for kid, name in enumerate(lhc.KERNEL_NAMES):
        t, n, _ = ctx.profile_read(kid)
        if n:
            kern[name] = {"ms_per_step": t, "launches_per_step": n}
    _line(args, B.METRIC, units * args.steps / (ms / 1e3), ms / args.steps,
          "baryon 3pt 32^3x64, eps-eps spectator of two complex64 propagators, N_r=32, t_f in {8,10,12,14}, "
          "123 momenta (|k|^2<=9, |k_j|<=3), insertion on slices 0..t_f, combine for 4 structures",
          {"clocks": clk, "roofline": _roofline(ctx), "kernels": kern, "units_per_step": units, "gpu_launches": nl})
    ctx.close()


# --------------------------------------------------------------------------- batched

def run_batched(args, dev, g):
    from paper_1711_02384_gb300 import inputs
    L, T, NR, DTS = 32, 64, 16, (8, 10, 12)
    V3 = L ** 3
    src = inputs.source_positions(4000, L, T, 16)
    rng = np.random.default_rng(4001)
    S = _rand((T, V3, 12, 12), torch.complex64, dev, g)
    psi = _rand((NR, T, V3, 12), torch.complex64, dev, g)
    eta = _rand((NR, V3, 12), torch.complex64, dev, g)
    ctx = lhc.Context(0)
    ctx.set_tuning(not args.no_tune)   # tuned in the first, uncaptured pass over the calls
    jobs = []
    for s_i in range(16):
        for dt in DTS:
            n2 = int(rng.integers(4, 17))
            k = lhc.momenta(n2)
            nq = len(k)
            r = [int(v) for v in src[s_i]]
            t0 = r[3]
            jobs.append(dict(r=r, t0=t0, dt=dt, k=k, nq=nq,
                             oi=torch.empty((dt + 1, nq, NR, 192), dtype=torch.complex128, device=dev),
                             om=torch.empty((nq, NR, 192), dtype=torch.complex128, device=dev),
                             ob=torch.empty((nq, NR, 3072), dtype=torch.complex128, device=dev)))
    stream = torch.cuda.Stream(dev)

    def calls():
        for j in jobs:
            ctx.insertion(S, psi, j["t0"], j["t0"] + j["dt"], j["r"], j["k"], prec=args.prec, out=j["oi"],
                          stream=stream.cuda_stream)
            ts = (j["t0"] + j["dt"]) % T
            ctx.spectator(S, eta, ts, j["r"], j["k"], prec=args.prec, out=j["om"], stream=stream.cuda_stream)
            ctx.spectator(S, eta, ts, j["r"], j["k"], prec=args.prec, GB=S, out=j["ob"], stream=stream.cuda_stream)

    # the same calls as one batch: one fused launch per part kind and momentum-chunk width
    batch = []
    for j in jobs:
        ts = (j["t0"] + j["dt"]) % T
        batch.append(dict(part="ins", S=S, vec=psi, t_lo=j["t0"], t_hi=j["t0"] + j["dt"], r=j["r"], k=j["k"], out=j["oi"]))
        batch.append(dict(part="spec", S=S, vec=eta, t_lo=ts, t_hi=ts, r=j["r"], k=j["k"], out=j["om"]))
        batch.append(dict(part="baryon", S=S, GB=S, vec=eta, t_lo=ts, t_hi=ts, r=j["r"], k=j["k"], out=j["ob"]))
    use_batch = args.prec == "mixed"

    def step_calls():
        if use_batch:
            ctx.batch(batch, stream=stream.cuda_stream)
        else:
            calls()

    with torch.cuda.stream(stream):
        calls()                      # tunes the launch shapes, builds the phase tables, sizes the workspace
        step_calls()
        torch.cuda.synchronize(dev)
        # the same calls one by one, captured in a graph of their own, for comparison
        ctx.set_projection("gemm")   # as the batch: the tensor-core projection for every call
        g1 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g1, stream=stream):
            calls()
        ms1, clk1, _ = _timed(lambda: g1.replay(), args.steps, args.warmup, dev, stream=stream, ctx=ctx)
        del g1
        graph = torch.cuda.CUDAGraph()
        n0 = lhc.launch_count()
        with torch.cuda.graph(graph, stream=stream):
            step_calls()
        n_graph = lhc.launch_count() - n0
        # graph.replay() launches on the current stream: keep it, and the events, on `stream`
        ms, clk, _ = _timed(lambda: graph.replay(), args.steps, args.warmup, dev, stream=stream, ctx=ctx)
        # one replay against the same calls issued directly: identical bits expected
        outs = [o for j in jobs for o in (j["oi"], j["om"], j["ob"])]
        for o in outs:
            o.zero_()
        graph.replay()
        torch.cuda.synchronize(dev)
        from_graph = [o.clone() for o in outs]
        ctx.profile(True)
        calls()
        torch.cuda.synchronize(dev)
        ctx.profile(False)
        same = all(torch.equal(a, b) for a, b in zip(from_graph, outs))
        del from_graph
    units = sum(V3 * NR * j["nq"] * (j["dt"] + 3) for j in jobs)
    _line(args, B.METRIC, units * args.steps / (ms / 1e3), ms / args.steps,
          "batched 32^3x64, 16 sources x t_f-t_0 in {8,10,12}, N_r=16, meson insertion + meson and baryon "
          "spectators, per-job momentum sets |k|^2<=4..16 (33..257), one CUDA graph per step"
          + (", all 144 calls in one lhc_batch (one persistent fused launch per part kind and chunk width)"
             if use_batch else ""),
          {"clocks": clk, "roofline": _roofline(ctx), "units_per_step": units, "jobs": len(jobs),
           "gpu_launches": n_graph * args.steps, "kernels_per_graph": n_graph,
           "graph_replay_equals_direct_calls": same,
           "one_by_one": {"ms_per_step": ms1 / args.steps, "clocks": clk1},
           "speedup_batch_over_one_by_one": (ms1 / ms) if use_batch else None})
    ctx.close()


# --------------------------------------------------------------------------- serve

def serve_stream(dev, g, prec, njobs=200, lat_shapes=((16, 32), (24, 48), (32, 64), (48, 96)),
                 fp64_small=0, seed=5000):
    """A Poisson stream of meson three-point jobs (spectator + insertion) through the job
    server: resident complex64 propagators on every lattice of `lat_shapes`, N_r in
    {8, 16, 32}, |k|^2 <= 4..16, t_f - t_0 in {8, 10, 12}, 4 slots, 150 GB budget.  The
    capacity is measured first (all jobs submitted at once), then the jobs arrive at 0.7 x
    capacity.  Returns the served throughput, the latency percentiles (submit to
    poll-visible completion), the most jobs that ran at once (from the jobs' start and
    done times), and with fp64_small > 0 the plain FP64 path one job at a time on that
    many jobs of the two smaller lattices, beside the mixed path on the same jobs."""
    NRMAX = 32
    ctx = lhc.Context(dev.index, hbm_budget=150 << 30)
    ctx.serve_start(slots=4)
    lats = []
    for L, T in lat_shapes:
        V3 = L ** 3
        S = _rand((T, V3, 12, 12), torch.complex64, dev, g)
        lats.append(dict(L=L, T=T, V3=V3, S=S, h=ctx.prop_register(S),
                         psi=_rand((NRMAX, T, V3, 12), torch.complex64, dev, g),
                         eta=_rand((NRMAX, V3, 12), torch.complex64, dev, g)))
    rng = np.random.default_rng(seed)
    specs = []
    for _ in range(njobs):
        li = int(rng.integers(len(lats)))
        specs.append(dict(li=li, n_r=int(rng.choice([8, 16, 32])), n2=int(rng.integers(4, 17)),
                          dt=int(rng.choice([8, 10, 12]))))
    kcache = {}
    for sp in specs:
        kcache.setdefault(sp["n2"], lhc.momenta(sp["n2"]))

    def units(sp):
        return lats[sp["li"]]["V3"] * sp["n_r"] * len(kcache[sp["n2"]]) * (sp["dt"] + 2)

    def submit(sp, p):
        la = lats[sp["li"]]
        k = kcache[sp["n2"]]
        nq = len(k)
        oi = torch.empty((sp["dt"] + 1, nq, sp["n_r"], 192), dtype=torch.complex128, device=dev)
        os_ = torch.empty((nq, sp["n_r"], 192), dtype=torch.complex128, device=dev)
        jid = ctx.submit(lhc.JOB_THREEPT, la["h"], k, prec=p, psi=la["psi"], eta=la["eta"], n_r=sp["n_r"],
                         t_lo=0, t_hi=sp["dt"], t_sink=sp["dt"], out_ins=oi, out_spec=os_)
        return jid, (oi, os_)

    # warm-up: one job per (lattice, momentum set) shape builds phase tables and workspaces
    seen, warm = set(), []
    for sp in specs:
        key = (sp["li"], sp["n2"])
        if key not in seen:
            seen.add(key)
            warm.append(submit(sp, prec))
    for jid, _ in warm:
        ctx.wait(jid, 600000)
    torch.cuda.synchronize(dev)

    # capacity: everything submitted at once
    t0 = time.perf_counter()
    sub = [submit(sp, prec) for sp in specs]
    for jid, _ in sub:
        ctx.wait(jid, 600000)
    cap_s = time.perf_counter() - t0
    del sub
    total_units = sum(units(sp) for sp in specs)
    cap_jobs = njobs / cap_s

    # Poisson arrivals at 70 % of capacity
    lam = 0.7 * cap_jobs
    gaps = rng.exponential(1.0 / lam, njobs)
    clocks = B.Clocks(B.nvsmi_id(dev.index), window="served stream")
    clocks.start()
    n0 = lhc.launch_count()
    t0 = time.perf_counter()
    live, t_next = [], t0
    for sp, gap in zip(specs, gaps):
        t_next += gap
        while time.perf_counter() < t_next:
            time.sleep(min(0.0005, max(0.0, t_next - time.perf_counter())))
        live.append(submit(sp, prec))
    for jid, _ in live:
        ctx.wait(jid, 600000)
    stream_s = time.perf_counter() - t0
    clk = clocks.stop()
    n_launch = lhc.launch_count() - n0
    lat_ms, spans = [], []
    for jid, _ in live:
        ts, tst, td = ctx.job_times(jid)
        lat_ms.append((td - ts) * 1e3)
        spans.append((tst, td))
    del live
    # the most jobs running at once: +1 at each start, -1 at each completion
    ev = sorted([(a, 1) for a, _ in spans] + [(b, -1) for _, b in spans], key=lambda e: (e[0], e[1]))
    run = peak = 0
    for _, d in ev:
        run += d
        peak = max(peak, run)
    out = {"value": total_units / stream_s, "unit": UNIT, "jobs": njobs, "stream_s": stream_s,
           "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                          "max": float(np.max(lat_ms))},
           "capacity": {"jobs_per_s": cap_jobs, "value": total_units / cap_s},
           "arrival_rate_jobs_per_s": lam, "max_concurrent_jobs": peak, "clocks": clk, "gpu_launches": n_launch,
           "lattices": [f"{L}^3x{T}" for L, T in lat_shapes]}
    if fp64_small:
        # plain FP64, one job at a time, on jobs of the two smaller lattices (FP64 on the
        # larger ones takes minutes per job); the mixed path one at a time on the same jobs
        small = [sp for sp in specs if sp["li"] <= 1][:fp64_small]
        res = {}
        for p in ("fp64", prec):
            t0 = time.perf_counter()
            for sp in small:
                jid, _ = submit(sp, p)
                ctx.wait(jid, 600000)
            res[p] = sum(units(sp) for sp in small) / (time.perf_counter() - t0)
        out["one_at_a_time_small_jobs"] = {"fp64": res["fp64"], prec: res[prec], "unit": UNIT, "jobs": len(small)}
    ctx.close()
    return out


def run_serve(args, dev, g):
    sv = serve_stream(dev, g, args.prec, njobs=200, fp64_small=6)
    _line(args, B.METRIC + " (served stream)", sv["value"], sv["stream_s"] * 1e3 / sv["jobs"],
          "served: 200 Poisson-arriving meson 3pt jobs (spectator + insertion) on 16^3x32, 24^3x48, 32^3x64, "
          "48^3x96 complex64 resident propagators, N_r in {8,16,32}, |k|^2<=4..16, t_f-t_0 in {8,10,12}, "
          "4 slots, 150 GB budget, arrival rate 0.7 x measured capacity",
          {k: v for k, v in sv.items() if k not in ("value", "unit", "stream_s")})


# --------------------------------------------------------------------------- mom1

def run_mom1(args, dev, g):
    L, NR, TFS = 24, 16, (8, 10, 12)
    V3 = L ** 3
    S = _rand((13, V3, 12, 12), torch.complex128, dev, g)
    psis = [_rand((NR, 13, V3, 12), torch.complex128, dev, g) for _ in TFS]
    etas = [_rand((NR, V3, 12), torch.complex128, dev, g) for _ in TFS]
    ctx = lhc.Context(0)
    r = (0, 0, 0, 0)
    out = {}
    for name, k in (("nq1", np.zeros((1, 3), dtype=np.int32)), ("nq93", lhc.momenta(8))):
        nq = len(k)
        oi = [torch.empty((tf + 1, nq, NR, 192), dtype=torch.complex128, device=dev) for tf in TFS]
        osp = [torch.empty((nq, NR, 192), dtype=torch.complex128, device=dev) for _ in TFS]

        def step():
            for j, tf in enumerate(TFS):
                ctx.insertion(S, psis[j], 0, tf, r, k, prec=args.prec, out=oi[j])
                ctx.spectator(S, etas[j], tf, r, k, prec=args.prec, out=osp[j])

        ms, clk, nl = _timed(step, args.steps, args.warmup, dev, ctx=ctx)
        out[name] = {"ms_per_step": ms / args.steps, "nq": nq, "gpu_launches": nl, "clocks": clk,
                     "value": sum(tf + 2 for tf in TFS) * V3 * NR * nq * args.steps / (ms / 1e3)}
    ctx.close()
    print(json.dumps({"metric": "step time at 93 momenta / step time at 1 momentum (meson 24^3x48)",
                      "value": out["nq93"]["ms_per_step"] / out["nq1"]["ms_per_step"], "unit": "ratio",
                      "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "f32+f16x2->f32 (mixed)" if args.prec == "mixed" else "f64",
                      "data": "synthetic (seeded random device tensors)",
                      "config": {"workload": "meson 24^3x48 insertion+spectator, 1 vs 93 momenta",
                                 "precision": args.prec}, "runs": out}))


# --------------------------------------------------------------------------- allmom

def run_allmom(args, dev, g):
    L, NR, NT = 16, 16, 4
    V3 = L ** 3
    lo = -(L // 2)
    k = np.array([(x, y, z) for z in range(lo, lo + L) for y in range(lo, lo + L) for x in range(lo, lo + L)],
                 dtype=np.int32)
    nq = len(k)
    S = _rand((NT + 1, V3, 12, 12), torch.complex128, dev, g)
    psi = _rand((NR, NT + 1, V3, 12), torch.complex128, dev, g)
    eta = _rand((NR, V3, 12), torch.complex128, dev, g)
    oi = torch.empty((NT, nq, NR, 192), dtype=torch.complex128, device=dev)
    osp = torch.empty((nq, NR, 192), dtype=torch.complex128, device=dev)
    ctx = lhc.Context(0)
    r = (3, 5, 7, 0)
    units = (NT + 1) * V3 * NR * nq
    out = {}
    for name, prec, mode, steps in (("dft_fp64", "fp64", "dft", args.steps), ("dft_mixed", "mixed", "dft", args.steps),
                                    ("gemm_mixed", "mixed", "gemm", args.steps), ("gemm_fp64", "fp64", "gemm", 1)):
        ctx.set_projection(mode)

        def step():
            ctx.insertion(S, psi, 0, NT - 1, r, k, prec=prec, out=oi)
            ctx.spectator(S, eta, NT, r, k, prec=prec, out=osp)

        ms, clk, nl = _timed(step, steps, 1 if name == "gemm_fp64" else args.warmup, dev, ctx=ctx)
        out[name] = {"ms_per_step": ms / steps, "value": units * steps / (ms / 1e3), "gpu_launches": nl,
                     "clocks": clk}
    ctx.close()
    print(json.dumps({"metric": "site*noise*mom contractions/s (all momenta)", "value": out["dft_fp64"]["value"],
                      "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": out["dft_fp64"]["ms_per_step"], "dtype": "f64",
                      "data": "synthetic (seeded random device tensors)",
                      "config": {"workload": "meson insertion (4 slices) + spectator on 16^3, 16 noises, all 4096 "
                                             "momenta, complex128; projection by DFT vs direct",
                                 "l2": "inputs of every step larger than L2 (129 MB)"},
                      "runs": out,
                      "dft_vs_gemm_fp64": out["gemm_fp64"]["ms_per_step"] / out["dft_fp64"]["ms_per_step"],
                      "dft_vs_gemm_mixed": out["gemm_mixed"]["ms_per_step"] / out["dft_fp64"]["ms_per_step"],
                      "mixed_dft_vs_mixed_gemm": out["gemm_mixed"]["ms_per_step"] / out["dft_mixed"]["ms_per_step"]}))


# --------------------------------------------------------------------------- paper

def run_paper(args, dev, g):
    L, NR, D = 32, 50, 10
    V3 = L ** 3
    nsl = 2 * D + 1                                   # slab of slices x4' .. x4'' (source in the middle)
    k = lhc.momenta(8)
    nq = len(k)
    S = _rand((nsl, V3, 12, 12), torch.complex128, dev, g)
    psi = _rand((NR, nsl, V3, 12), torch.complex128, dev, g)
    eta_b = _rand((NR, V3, 12), torch.complex128, dev, g)     # the noise on the backward sink slice
    eta_f = _rand((NR, V3, 12), torch.complex128, dev, g)     # and on the forward one
    g16 = torch.from_numpy(B.gamma_sets()[0]).to(dev)
    g4 = torch.from_numpy(B.gamma_sets()[1]).to(dev)
    Ws = _rand((4, 4, 4, 4), torch.complex128, dev, g)
    Wc = _rand((4, 4, 4, 4), torch.complex128, dev, g)
    ctx = lhc.Context(0)
    ctx.set_tuning(not args.no_tune)
    r = (0, 0, 0, D)                                  # slab index of the source time (t = 30 of 96)
    oi = torch.empty((nsl, nq, NR, 192), dtype=torch.complex128, device=dev)
    om = [torch.empty((nq, NR, 192), dtype=torch.complex128, device=dev) for _ in range(2)]
    ob = [torch.empty((nq, NR, 3072), dtype=torch.complex128, device=dev) for _ in range(2)]
    cm = [torch.empty((D + 1, 16, nq, nq), dtype=torch.complex128, device=dev) for _ in range(2)]
    cb = [torch.empty((D + 1, 4, nq, nq), dtype=torch.complex128, device=dev) for _ in range(2)]

    def step():
        ctx.insertion(S, psi, 0, nsl - 1, r, k, prec=args.prec, out=oi)   # both directions in one call
        for d, (ts, eta) in enumerate(((0, eta_b), (nsl - 1, eta_f))):
            ctx.spectator(S, eta, ts, r, k, prec=args.prec, out=om[d])
            ctx.spectator(S, eta, ts, r, k, prec=args.prec, GB=S, out=ob[d])
            ins = oi[0:D + 1] if d == 0 else oi[D:nsl]
            ctx.combine(om[d], ins, g16, g4, g16, prec=args.prec, out=cm[d])
            ctx.combine(ob[d], ins, Ws, g4[:4], Wc, prec=args.prec, out=cb[d])

    ms, clk, nl = _timed(step, args.steps, args.warmup, dev, ctx=ctx)
    units = (nsl + 4) * V3 * NR * nq
    ctx.close()
    _line(args, B.METRIC, units * args.steps / (ms / 1e3), ms / args.steps,
          "the paper's measurement shape: 32^3x96, source t=30, sinks t=20 and t=40 (forward and backward), "
          "50 noises on both sink slices, 93 momenta at sink and insertion, one insertion call over t=20..40, "
          "meson and baryon spectators, meson combine (16 structures) and baryon combine (4) per direction, "
          "complex128 inputs",
          {"clocks": clk, "units_per_step": units, "gpu_launches": nl,
           "ms_per_configuration": ms / args.steps,
           "paper_context": "about 575 s per configuration on 8 KNL nodes (QPACE3) for the paper's whole "
                            "measurement with k^2, k'^2 <= 8; other hardware, and its scope (I/O, smearing) differs"})


# --------------------------------------------------------------------------- extras

def run_extras(args, dev, g):
    ctx = lhc.Context(0)
    out = {}
    # the open-spin combine's sweep over all 16 x 16 x 16 Dirac structures on one slice
    nq, NR = 93, 16
    spec = _rand((nq, NR, 192), torch.complex128, dev, g)
    ins = _rand((1, nq, NR, 192), torch.complex128, dev, g)
    g16 = torch.from_numpy(B.gamma_sets()[0]).to(dev)
    res = torch.empty((1, 16, 16, nq, nq, 4, 4), dtype=torch.complex128, device=dev)
    for prec in ("mixed", "fp64"):
        ms, clk, nl = _timed(lambda: ctx.combine_open(spec, ins, g16, g16, prec=prec, out=res), args.steps,
                             args.warmup, dev, ctx=ctx)
        out["open_combine_" + prec] = {"ms_per_sweep": ms / args.steps,
                                       "correlators_per_s": 16 ** 3 * nq * nq * args.steps / (ms / 1e3),
                                       "clocks": clk}
    # the baryon open combine: 4 sink structures x 16 insertion Gammas, source spins open
    bspec = _rand((nq, NR, 3072), torch.complex128, dev, g)
    w4 = _rand((4, 4, 4, 4), torch.complex128, dev, g)
    bres = torch.empty((1, 4, 16, nq, nq, 4, 4, 4), dtype=torch.complex128, device=dev)
    for prec in ("mixed", "fp64"):
        ms, clk, nl = _timed(lambda: ctx.combine_open_baryon(bspec, ins, w4, g16, prec=prec, out=bres), args.steps,
                             args.warmup, dev, ctx=ctx)
        out["open_baryon_combine_" + prec] = {"ms_per_call": ms / args.steps, "sink_structures": 4,
                                              "insertion_gammas": 16,
                                              "open_blocks_per_s": 4 * 16 * nq * nq * args.steps / (ms / 1e3),
                                              "clocks": clk}
    del bspec, bres
    # free-field Wilson-Dirac solves: 12 point sources on 16^3 x 32
    from paper_1711_02384_gb300 import inputs
    L, T = 16, 32
    src = torch.zeros((12, T, L ** 3, 12), dtype=torch.complex128, device=dev)
    for sc in range(12):
        src[sc, 0, 0, sc] = 1.0
    gam = inputs.dirac_matrices()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sol, it, rr = ctx.wilson_solve(src, 0.3, gam, tol=1e-12)
    torch.cuda.synchronize(dev)
    out["free_solve_16c32"] = {"ms": 1e3 * (time.perf_counter() - t0), "rhs": 12, "iterations": it,
                               "relative_residual": rr, "mass": 0.3}
    ctx.close()
    print(json.dumps({"metric": "open-spin combine sweep and free-field solve", "unit": "ms", "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
                      "data": "synthetic (seeded random device tensors)",
                      "config": {"workload": "Dirac sweep 16x16x16 over one slice (93x93 momenta, 16 noises); "
                                             "baryon open combine, 4 W_snk x 16 Gamma_ins, (a1, a2, b) open; "
                                             "12 point sources, free Wilson-Dirac, 16^3x32, m = 0.3"},
                      "runs": out}))


# --------------------------------------------------------------------------- smallcalls

def run_smallcalls(args, dev, g):
    """Many small calls: 48 source positions on a 16^3 x 32 lattice, each an insertion over
    3 slices and a meson spectator with 4 noises and its own momentum set (|k|^2 <= 1..8,
    7 to 93 momenta, chunk widths 8 to 48).  A single call launches fewer CTAs than the GPU
    has SMs, so one by one the GPU stays partly empty; the batch runs each part kind's calls
    in persistent launches (one per part kind and chunk width).  Both forms are captured in
    CUDA graphs and replayed."""
    from paper_1711_02384_gb300 import inputs
    L, T, NR, NSRC = 16, 32, 4, 48
    V3 = L ** 3
    src = inputs.source_positions(4100, L, T, NSRC)
    rng = np.random.default_rng(4101)
    S = _rand((T, V3, 12, 12), torch.complex64, dev, g)
    psi = _rand((NR, T, V3, 12), torch.complex64, dev, g)
    eta = _rand((NR, V3, 12), torch.complex64, dev, g)
    ctx = lhc.Context(0)
    ctx.set_tuning(False)          # the heuristic launch shapes, the same in both forms
    ctx.set_projection("gemm")     # as the batch: the tensor-core projection for every call
    calls = []
    for s_i in range(NSRC):
        k = lhc.momenta(int(rng.integers(1, 9)))
        r = [int(v) for v in src[s_i]]
        nq = len(k)
        ts = (r[3] + 2) % T
        calls.append(dict(part="ins", S=S, vec=psi, t_lo=r[3], t_hi=r[3] + 2, r=r, k=k,
                          out=torch.empty((3, nq, NR, 192), dtype=torch.complex128, device=dev)))
        calls.append(dict(part="spec", S=S, vec=eta, t_lo=ts, t_hi=ts, r=r, k=k,
                          out=torch.empty((nq, NR, 192), dtype=torch.complex128, device=dev)))
    stream = torch.cuda.Stream(dev)

    def one_by_one():
        for c in calls:
            if c["part"] == "ins":
                ctx.insertion(c["S"], c["vec"], c["t_lo"], c["t_hi"], c["r"], c["k"], prec="mixed", out=c["out"],
                              stream=stream.cuda_stream)
            else:
                ctx.spectator(c["S"], c["vec"], c["t_lo"], c["r"], c["k"], prec="mixed", out=c["out"],
                              stream=stream.cuda_stream)

    def batched():
        ctx.batch(calls, stream=stream.cuda_stream)

    res = {}
    with torch.cuda.stream(stream):
        for name, fn in (("one_by_one", one_by_one), ("batch", batched)):
            fn()                       # phase tables, workspace
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            n0 = lhc.launch_count()
            with torch.cuda.graph(graph, stream=stream):
                fn()
            nk = lhc.launch_count() - n0
            ms, clk, _ = _timed(lambda: graph.replay(), args.steps, args.warmup, dev, stream=stream, ctx=ctx)
            res[name] = {"ms_per_step": ms / args.steps, "kernels_per_graph": nk, "clocks": clk}
            if name == "one_by_one":
                ref = [c["out"].clone() for c in calls]
        same = all(torch.equal(c["out"], r) for c, r in zip(calls, ref))
    units = sum(V3 * NR * len(c["k"]) * (c["t_hi"] - c["t_lo"] + 1) for c in calls)
    ms = res["batch"]["ms_per_step"]
    _line(args, B.METRIC, units / (ms / 1e3), ms,
          "many small calls: 48 sources on 16^3x32, each a 3-slice insertion + meson spectator with 4 noises and "
          "its own momentum set (|k|^2<=1..8, 7..93 momenta), complex64; the batch (one persistent launch per "
          "part kind and chunk width) against the same calls one by one, both replayed from CUDA graphs",
          {"units_per_step": units, "calls": len(calls), "one_by_one": res["one_by_one"], "batch": res["batch"],
           "speedup_batch_over_one_by_one": res["one_by_one"]["ms_per_step"] / ms,
           "batch_equals_one_by_one": same, "gpu_launches": res["batch"]["kernels_per_graph"] * args.steps,
           "clocks": res["batch"]["clocks"]})
    ctx.close()


def run(args):
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(1711)
    {"baryon32": run_baryon32, "batched": run_batched, "serve": run_serve, "mom1": run_mom1,
     "allmom": run_allmom, "paper": run_paper, "extras": run_extras,
     "smallcalls": run_smallcalls}[args.workload](args, dev, g)
