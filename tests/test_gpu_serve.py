"""The job server: continuous batching with resident propagators and HBM-budget
admission.  A job's result is the same alone and in a mix; budgets, cancellation and
polling behave as documented; bounded device waits report LHC_ETIMEOUT."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_job_inputs(L, T, n_r, seed, dtype=np.complex64):
    from paper_1711_02384_gb300 import inputs
    S = inputs.propagator(seed, L, T).astype(dtype)
    psi = inputs.solutions(seed + 1, L, T, n_r).astype(dtype)
    return S, psi


def test_mix_equals_alone_and_oracle():
    from oracle import contractions as OC
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import inputs, lhc
    with lhc.Context(0, hbm_budget=8 << 30) as ctx:
        ctx.serve_start(slots=4)
        lattices = [(4, 8, 4, 3), (6, 8, 2, 2), (8, 16, 8, 4), (5, 8, 3, 1)]   # L, T, n_r, n2max
        props, jobs_in = [], []
        for j, (L, T, n_r, n2) in enumerate(lattices):
            S, psi = make_job_inputs(L, T, n_r, 4000 + 10 * j)
            eta = inputs.noise(4005 + 10 * j, L, n_r, 5).astype(np.complex64)
            dS = dev(S)
            props.append((dS, ctx.prop_register(dS)))
            jobs_in.append((L, T, n_r, momenta(n2), S, dev(psi), dev(eta), psi, eta))

        def submit(j):
            L, T, n_r, k, S, dpsi, deta, psi, eta = jobs_in[j]
            nq = len(k)
            oi = torch.empty((6, nq, n_r, 192), dtype=torch.complex128, device="cuda")
            os_ = torch.empty((nq, n_r, 192), dtype=torch.complex128, device="cuda")
            jid = ctx.submit(lhc.JOB_THREEPT, props[j][1], k, r=(1, 0, 2, 0), psi=dpsi, eta=deta, t_lo=0, t_hi=5,
                             t_sink=5, out_ins=oi, out_spec=os_)
            return jid, oi, os_

        alone = []
        for j in range(len(jobs_in)):
            jid, oi, os_ = submit(j)
            ctx.wait(jid)
            alone.append((oi.clone(), os_.clone()))
        # the mix: every job three times, all submitted at once
        mix = [(j, submit(j)) for _ in range(3) for j in range(len(jobs_in))]
        for j, (jid, oi, os_) in mix:
            ctx.wait(jid)
            assert torch.equal(oi, alone[j][0]) and torch.equal(os_, alone[j][1]), f"job {j} differs in the mix"
        # and the results are right
        g5 = CS.g5_matrix()
        for j, (L, T, n_r, k, S, _, _, psi, eta) in enumerate(jobs_in):
            ref_i = OC.insertion(S[0:6].astype(complex), psi[:, 0:6].astype(complex), g5, (1, 0, 2), k, L)
            ref_s = OC.spectator_meson(S[5].astype(complex), eta.astype(complex), g5, (1, 0, 2), k, L)
            assert CS.block_err(alone[j][0].cpu().numpy(), ref_i, 2) < CS.MIXED_TOL
            assert CS.block_err(alone[j][1].cpu().numpy(), ref_s, 1) < CS.MIXED_TOL
        used, queued, running = ctx.serve_stats()
        assert queued == 0 and running == 0 and used > 0


def max_overlap(spans):
    """The most intervals [a, b] that contain one point in time."""
    ev = sorted([(a, 1) for a, _ in spans] + [(b, -1) for _, b in spans], key=lambda e: (e[0], e[1]))
    run = peak = 0
    for _, d in ev:
        run += d
        peak = max(peak, run)
    return peak


def test_admitted_jobs_overlap_on_the_device():
    """Continuous batching: jobs submitted together into four slots have their work in
    flight on the device at the same time.  Each job's device interval comes from timing
    events on its slot's stream (lhc_job_device_times); at least two intervals intersect,
    and so do the host intervals from admission to completion (lhc_job_times).  The mixed
    results still equal those of the same job run alone, bit for bit."""
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    L, T, n_r = 16, 16, 8
    S, psi = make_job_inputs(L, T, n_r, 4200)
    dS, dpsi = dev(S), dev(psi)
    k = momenta(4)
    nq = len(k)
    with lhc.Context(0) as ctx:
        ctx.serve_start(slots=4)
        h = ctx.prop_register(dS)

        def submit():
            out = torch.empty((8, nq, n_r, 192), dtype=torch.complex128, device="cuda")
            return ctx.submit(lhc.JOB_INSERTION, h, k, psi=dpsi, t_lo=0, t_hi=7, out_ins=out), out

        jid, alone = submit()
        ctx.wait(jid)
        jobs = [submit() for _ in range(8)]
        for jid, out in jobs:
            ctx.wait(jid)
            assert torch.equal(out, alone)
        dev_spans = [ctx.job_device_times(jid) for jid, _ in jobs]
        host_spans = [ctx.job_times(jid)[1:] for jid, _ in jobs]
        assert all(0.0 <= a <= b for a, b in dev_spans)
        print(f"[serve] most jobs in flight at once: device {max_overlap(dev_spans)}, host {max_overlap(host_spans)}")
        assert max_overlap(dev_spans) >= 2
        assert max_overlap(host_spans) >= 2


def test_budget_refusal_and_polling_and_cancel():
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    L, T, n_r = 16, 16, 8
    S, psi = make_job_inputs(L, T, n_r, 4100)
    dS, dpsi = dev(S), dev(psi)
    k = momenta(4)
    out = torch.empty((T, len(k), n_r, 192), dtype=torch.complex128, device="cuda")
    # a budget that holds the propagator but never the job's workspace
    with lhc.Context(0, hbm_budget=dS.numel() * 8 + (1 << 20)) as small:
        small.serve_start(slots=1)
        h = small.prop_register(dS)
        with pytest.raises(lhc.LhcError) as e:
            small.submit(lhc.JOB_INSERTION, h, k, psi=dpsi, t_lo=0, t_hi=T - 1, out_ins=out)
        assert e.value.status == lhc.EBUDGET
    with lhc.Context(0) as ctx:
        ctx.serve_start(slots=1)
        h = ctx.prop_register(dS)
        first = ctx.submit(lhc.JOB_INSERTION, h, k, prec="fp64", psi=dpsi, t_lo=0, t_hi=T - 1, out_ins=out)
        out2 = torch.empty_like(out)
        second = ctx.submit(lhc.JOB_INSERTION, h, k, psi=dpsi, t_lo=0, t_hi=T - 1, out_ins=out2)
        assert ctx.cancel(second) == lhc.OK                 # one slot: still queued behind the first
        status, state = ctx.poll(second)
        assert status == lhc.OK and state == lhc.JOB_CANCELED
        assert ctx.wait_status(second) == lhc.ECANCELED
        ctx.wait(first)
        status, state = ctx.poll(first)
        assert status == lhc.OK and state == lhc.JOB_DONE
        ts, t0, t1 = ctx.job_times(first)
        assert ts <= t0 <= t1
        with pytest.raises(lhc.LhcError):
            ctx.prop_release(12345)


def test_bounded_device_wait_reports_timeout():
    from paper_1711_02384_gb300 import lhc
    with lhc.Context(0) as ctx:
        t0 = time.time()
        assert ctx.selftest_timeout(200000) == lhc.ETIMEOUT
        assert time.time() - t0 < 30
        # the context stays usable
        assert ctx.selftest_timeout(1000) == lhc.ETIMEOUT
        ctx.sync()
