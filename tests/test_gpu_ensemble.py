"""The batched ensemble (cams_ensemble_solve): independent realisations run
concurrently, each on a stream of a worker thread.  Every member's result
must be bit-for-bit the one-at-a-time cams_solve result (no kernel depends on
the stream or on what runs beside it), and the small members are held to
the FP64 oracle like every other solve (1e-6 relative L-infinity for the
mixed-precision preconditioner, Newton counts within one)."""
import numpy as np
import pytest

import oracle
from _cases import gpu_handle, make_case
from workloads import ensemble_members

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cams():
    from paper_1705_05783_gb300 import cams
    return cams


def _small_members(k, precision=1):
    ms = [w for w in ensemble_members(64, precision=precision) if w.n_cells <= 100_000]
    return ms[:k]


def _cases(members):
    return [make_case(w=w, seed=w.seeds[0]) for w in members]


def _handles(cams, cases):
    hs, bcs, keep = [], [], []
    for c in cases:
        h, bc, kp = gpu_handle(c)
        hs.append(h); bcs.append(bc); keep.append(kp)
    return hs, bcs, keep


def _sequential(cams, hs, bcs, cases):
    out = []
    for h, bc, c in zip(hs, bcs, cases):
        p = c.inp["p0"].copy()
        st = cams.cams_solve(h, c.inp["p0"].copy(), c.inp["dt"], bc, p)
        out.append((p, st.newton_its, st.cams_its))
    return out


def _ensemble(cams, hs, bcs, cases, workers):
    pn = [c.inp["p0"].copy() for c in cases]
    ps = [c.inp["p0"].copy() for c in cases]
    status, st = cams.cams_ensemble_solve(hs, pn, [c.inp["dt"] for c in cases], bcs, ps, workers)
    return status, [(p, s.newton_its, s.cams_its) for p, s in zip(ps, st)]


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("workers", [1, 4])
def test_ensemble_equals_one_at_a_time(cams, precision, workers):
    cases = _cases(_small_members(6, precision))
    hs, bcs, keep = _handles(cams, cases)
    try:
        seq = _sequential(cams, hs, bcs, cases)
        status, ens = _ensemble(cams, hs, bcs, cases, workers)
        assert status == [cams.CAMS_OK] * len(cases)
        for (p1, n1, c1), (p2, n2, c2) in zip(seq, ens):
            assert np.array_equal(p1, p2)
            assert (n1, c1) == (n2, c2)
    finally:
        for h in hs:
            cams.cams_destroy(h)


def test_ensemble_members_match_oracle(cams):
    cases = _cases(_small_members(3))
    hs, bcs, keep = _handles(cams, cases)
    try:
        status, ens = _ensemble(cams, hs, bcs, cases, 3)
    finally:
        for h in hs:
            cams.cams_destroy(h)
    assert status == [cams.CAMS_OK] * 3
    for c, (p, n, _) in zip(cases, ens):
        q, sto = oracle.run(c.pb, c.opt, c.inp["p0"], c.inp["dt"], 1)
        assert np.abs(p - q).max() < 1e-6 * np.abs(q).max()
        assert abs(n - sto[0].newton_its) <= 1


def test_ensemble_reports_each_members_status(cams):
    """A member with a bad argument fails alone; the others still run and
    give their one-at-a-time results; the call returns that member's code."""
    cases = _cases(_small_members(4))
    hs, bcs, keep = _handles(cams, cases)
    try:
        seq = _sequential(cams, hs, bcs, cases)
        pn = [c.inp["p0"].copy() for c in cases]
        ps = [c.inp["p0"].copy() for c in cases]
        dts = [c.inp["dt"] for c in cases]
        dts[2] = -1.0
        status, st = cams.cams_ensemble_solve(hs, pn, dts, bcs, ps, 2)
        assert status[2] == cams.CAMS_EINVAL
        for k in (0, 1, 3):
            assert status[k] == cams.CAMS_OK
            assert np.array_equal(ps[k], seq[k][0])
    finally:
        for h in hs:
            cams.cams_destroy(h)


def test_ensemble_rejects_a_repeated_handle(cams):
    cases = _cases(_small_members(2))
    hs, bcs, keep = _handles(cams, cases)
    try:
        ps = [c.inp["p0"].copy() for c in cases]
        with pytest.raises(cams.CamsError) as e:
            cams.cams_ensemble_solve([hs[0], hs[0]], ps, [1.0, 1.0], [bcs[0], bcs[0]], ps)
        assert e.value.code == cams.CAMS_EINVAL
    finally:
        for h in hs:
            cams.cams_destroy(h)
