"""Host-side parts of the learned-surrogate trainer (no GPU): the parameter
layout agrees with the library's size, the initialisation is He-uniform with
zero biases, the stored parameters fit the layout, and the training fields
are seeded apart from the workloads' fields."""
import numpy as np

from paper_1705_05783_gb300 import cams, surrogate


def test_parameter_layout_and_initialisation():
    off = surrogate.offsets()
    assert len(off) == len(surrogate.LAYERS) == 4
    total = 0
    for (ci, co), (ow, ob) in zip(surrogate.LAYERS, off):
        assert ow == total and ob - ow == co * ci * 27
        total = ob + co
    assert total == cams.CAMS_NET_PARAMS
    p = surrogate.init_params(3)
    assert p.dtype == np.float32 and p.shape == (cams.CAMS_NET_PARAMS,)
    for (ci, co), (ow, ob) in zip(surrogate.LAYERS, off):
        lim = np.sqrt(6.0 / (27 * ci))
        w = p[ow:ob]
        assert np.all(np.abs(w) <= lim) and w.std() > 0.4 * lim      # uniform on [-lim, lim]
        assert np.all(p[ob:ob + co] == 0.0)                           # zero biases
    np.testing.assert_array_equal(surrogate.init_params(3), p)       # seeded


def test_stored_parameters_fit_the_layout():
    p = surrogate.load_params()
    assert p.shape == (cams.CAMS_NET_PARAMS,) and np.all(np.isfinite(p))


def test_training_fields_are_seeded_apart_from_the_workloads():
    from workloads import WORKLOADS
    fields = surrogate.training_fields(20)
    seeds = {w.seeds[0] for w in fields}
    assert len(seeds) == 20
    used = {s for w in WORKLOADS.values() for s in w.seeds}
    assert not seeds & used
    assert all(1.0 <= w.sigma <= 4.0 and w.precision == 0 for w in fields)
