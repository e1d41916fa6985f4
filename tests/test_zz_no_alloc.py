"""The allocation-free combine (lhc_combine_noalloc) through the C ABI.

It exists for callers that cannot let a library allocate device memory (a process whose
HBM is owned by another allocator, or host code that must not stall on cudaMalloc /
cudaFree, which can synchronize the device).  Its results must equal those of the
regular lhc_combine on the same inputs, on two calls in a row (the scratch array is
shared between calls and keeps the previous call's contents).  This file is collected
last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import _cases as CS

pytestmark = pytest.mark.gpu


def _noalloc(lib, kind, spec, ins, snk, gi, src, prec, out):
    np_, n_r = spec.shape[0], spec.shape[1]
    nt, nq = ins.shape[0], ins.shape[1]
    f = lib.lhc_combine_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p]
    st = torch.cuda.current_stream().cuda_stream
    return f(kind, spec.data_ptr(), np_, ins.data_ptr(), nq, n_r, nt, snk.data_ptr(), gi.data_ptr(),
             src.data_ptr(), gi.shape[0], prec, out.data_ptr(), st)


@pytest.mark.parametrize("kind", [0, 1])
def test_noalloc_matches_combine_twice(kind):
    from paper_1711_02384_gb300 import lhc
    lib = lhc.lib()
    dev = torch.device("cuda", 0)
    with lhc.Context(0) as ctx:
        for call, (seed, np_, nq, n_r, ng, nt) in enumerate([(21, 17, 23, 4, 3, 5), (22, 40, 600, 16, 8, 5)]):
            rng = np.random.default_rng(seed + 10 * kind)
            cols = 192 if kind == 0 else 3072
            c = lambda *s: torch.from_numpy(rng.standard_normal(s) + 1j * rng.standard_normal(s)).to(dev)
            spec, ins = c(np_, n_r, cols), c(nt, nq, n_r, 192)
            wshape = (4, 4) if kind == 0 else (4, 4, 4)
            snk, gi, src = c(ng, *wshape), c(ng, 4, 4), c(ng, *wshape)
            for prec, tol in ((0, CS.FP64_TOL), (1, CS.MIXED_TOL)):
                ref = ctx.combine(spec, ins, snk, gi, src, prec="fp64" if prec == 0 else "mixed")
                out = torch.full((nt, ng, np_, nq), float("nan"), dtype=torch.complex128, device=dev)
                status = _noalloc(lib, kind, spec, ins, snk, gi, src, prec, out)
                assert status == 0, lib.lhc_last_error()
                torch.cuda.synchronize()
                got, want = out.cpu().numpy(), ref.cpu().numpy()
                assert np.all(np.isfinite(got)), f"call {call}: unwritten outputs"
                for t in range(nt):
                    assert CS.corr_err(got[t], want[t]) < tol, (call, prec, t)


def test_noalloc_rejects_oversize_and_host_buffers():
    from paper_1711_02384_gb300 import lhc
    lib = lhc.lib()
    lib.lhc_last_error.restype = ctypes.c_char_p
    dev = torch.device("cuda", 0)
    # one insertion slice needs ng*(np+nq)*12*n_r*16 bytes: 16*(600+600)*12*16*16 > 32 MiB
    spec = torch.zeros((600, 16, 192), dtype=torch.complex128, device=dev)
    ins = torch.zeros((1, 600, 16, 192), dtype=torch.complex128, device=dev)
    g = torch.zeros((16, 4, 4), dtype=torch.complex128, device=dev)
    out = torch.zeros((1, 16, 600, 600), dtype=torch.complex128, device=dev)
    assert _noalloc(lib, 0, spec, ins, g, g, g, 0, out) == 1
    assert b"scratch" in lib.lhc_last_error()
    assert _noalloc(lib, 0, spec[:2].cpu(), ins[:, :2].cpu(), g.cpu(), g.cpu(), g.cpu(), 0,
                    out[:, :, :2, :2].cpu()) == 1
    if torch.cuda.device_count() > 1:   # a buffer of another GPU is refused, not read as peer memory
        other = spec[:2].to(torch.device("cuda", 1))
        assert _noalloc(lib, 0, other, ins[:, :2], g, g, g, 0, out[:, :, :2, :2]) == 1
        assert b"current device" in lib.lhc_last_error()
