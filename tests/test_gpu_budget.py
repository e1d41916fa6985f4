"""HBM budget: a context whose budget cannot hold a call's phase table and workspace
together refuses the call with LHC_EBUDGET; it never evicts a table the call has already
taken (which would leave the call reading freed memory).  A sweep of budgets from far
too small to ample, for the mixed path's tensor-core projection, its all-momenta
transform and the FP64 path: every call either is refused or gives the unbounded
result."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec,proj", [("mixed", "gemm"), ("mixed", "dft"), ("fp64", "gemm")])
def test_budget_sweep_refuses_or_matches(prec, proj):
    from oracle.momenta import momenta
    from paper_1711_02384_gb300 import lhc
    c = CS.Case(8, 4, 2, momenta(3), seed=5100, r=(1, 2, 3, 0))
    S, psi = dev(c.S), dev(c.psi)
    other = momenta(2)                        # a second list: its table is the one to evict

    def run(budget):
        with lhc.Context(0, hbm_budget=budget) as ctx:
            ctx.set_projection(proj)
            ctx.insertion(S, psi, 0, 1, c.r, other, prec=prec)
            out = ctx.insertion(S, psi, 0, 1, c.r, c.k, prec=prec)
            ctx.sync()
            return out.cpu().numpy()

    ref = run(0)
    assert CS.block_err(ref, c.ref_insertion(0, 1), 2) < (CS.MIXED_TOL if prec == "mixed" else CS.FP64_TOL)
    refused = matched = 0
    budget = 1 << 16
    while budget < (64 << 20):
        try:
            got = run(budget)
        except lhc.LhcError as e:
            assert e.status == lhc.EBUDGET, str(e)
            refused += 1
        else:
            # the same result up to the reduction order of another launch shape; a table
            # read after its eviction would be wrong at order one
            assert CS.block_err(got, ref, 2) < (CS.MIXED_TOL if prec == "mixed" else 1e-12), f"budget {budget}"
            matched += 1
        budget = int(budget * 1.12) + 4096
    assert refused > 0 and matched > 0
