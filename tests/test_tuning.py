"""Launch-shape autotuner of the mixed path: the table file format and loading (host
only), and on the GPU that a tuned call keeps parity with the oracle, records its shape,
persists it, that later calls of the shape reproduce the tuned call bit for bit, and that
tuning stops instead of recording a shape whose kernels gave up a bounded wait."""
import ctypes

import numpy as np
import pytest

from paper_1711_02384_gb300 import build as B


@pytest.fixture(scope="module")
def lhc():
    B.build()
    from paper_1711_02384_gb300 import lhc as m
    return m


def _rows(t, V3):
    return [tuple(int(x) for x in r) for r in t if r[2] == V3]


def test_table_file_loads(lhc, tmp_path):
    p = tmp_path / "shapes.txt"
    p.write_text("# comment\n0 0 999001 16 13 47  48 4  433.2\n\n2 1 999001 32 1 62  32 6  8000.0\n")
    assert lhc.tuning_load(p) == 2
    rows = _rows(lhc.tuning_table(), 999001)
    assert (0, 0, 999001, 16, 13, 47, 48, 4) in rows
    assert (2, 1, 999001, 32, 1, 62, 32, 6) in rows


def test_missing_file_is_an_empty_table(lhc, tmp_path):
    assert lhc.tuning_load(tmp_path / "none.txt") == 0


@pytest.mark.parametrize("line", ["0 0 999002 16 13 47 48", "0 0 999002 16 13 47 44 4 1.0", "5 0 999002 16 13 47 48 4 1.0"])
def test_malformed_lines_are_rejected(lhc, tmp_path, line):
    p = tmp_path / "bad.txt"
    p.write_text(line + "\n")
    with pytest.raises(lhc.LhcError):
        lhc.tuning_load(p)
    assert not _rows(lhc.tuning_table(), 999002)


@pytest.mark.gpu
def test_tuned_call_parity_persistence_and_reuse(lhc, tmp_path):
    torch = pytest.importorskip("torch")
    import _cases as CS
    from oracle.momenta import momenta
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    c = CS.Case(10, 4, 3, momenta(3), seed=1800, r=(2, 7, 1, 0))   # V3 = 1000, 16 representatives
    path = tmp_path / "shapes.txt"
    with lhc.Context(0) as ctx:
        ctx.set_tuning(True, path)
        before = len(lhc.tuning_table())
        gi = ctx.insertion(dev(c.S), dev(c.psi), 0, 3, c.r, c.k, prec="mixed")
        ctx.sync()
        assert len(lhc.tuning_table()) == before + 1
        row = [r for r in lhc.tuning_table() if r[0] == 0 and r[2] == 1000 and r[3] == 3]
        assert len(row) == 1 and row[0][4] == 4 and row[0][5] == 14
        assert CS.block_err(gi.cpu().numpy(), c.ref_insertion(0, 3), 2) < CS.MIXED_TOL
        # the file holds the entry; a later call of the shape reuses it (no new entry)
        assert " 1000 3 4 14 " in path.read_text()
        again = ctx.insertion(dev(c.S), dev(c.psi), 0, 3, c.r, c.k, prec="mixed")
        ctx.sync()
        assert len(lhc.tuning_table()) == before + 1
        assert torch.equal(gi, again)
    # another context without tuning finds the shape in the process-wide table
    with lhc.Context(0) as ctx2:
        third = ctx2.insertion(dev(c.S), dev(c.psi), 0, 3, c.r, c.k, prec="mixed")
        ctx2.sync()
        assert torch.equal(gi, third)


@pytest.mark.gpu
def test_autotune_stops_on_a_wait_that_gave_up(lhc):
    """A candidate whose kernels gave up a bounded wait would time as the fastest (every
    later wait gives up at once).  With the device error word set (the library's
    bounded-wait self-test, no fault), a tuned call must stop with LHC_ETIMEOUT and record
    no shape; after the sync reports the error, the same call tunes and runs."""
    torch = pytest.importorskip("torch")
    import _cases as CS
    from oracle.momenta import momenta
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    c = CS.Case(9, 4, 2, momenta(2), seed=1810, r=(1, 2, 3, 0))   # V3 = 729: a key no other test tunes
    with lhc.Context(0) as ctx:
        ctx.set_tuning(True)
        before = len(lhc.tuning_table())
        ctx.selftest_flag(1000)
        with pytest.raises(lhc.LhcError) as e:
            ctx.insertion(dev(c.S), dev(c.psi), 0, 1, c.r, c.k, prec="mixed")
        assert e.value.status == lhc.ETIMEOUT and "autotune" in str(e.value)
        assert len(lhc.tuning_table()) == before
        with pytest.raises(lhc.LhcError):
            ctx.sync()                                               # reports the flag, clears it
        gi = ctx.insertion(dev(c.S), dev(c.psi), 0, 1, c.r, c.k, prec="mixed")
        ctx.sync()
        assert len(lhc.tuning_table()) == before + 1
        assert CS.block_err(gi.cpu().numpy(), c.ref_insertion(0, 1), 2) < CS.MIXED_TOL
