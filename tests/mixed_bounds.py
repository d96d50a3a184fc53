"""Per-process bounds of the mixed-precision path (FP32 amplitudes and
external states, FP64 propagator denominators and helicity sum, FP16 hi+lo
colour contraction with FP32 accumulation) against the FP64 oracle.

Each bound is about ten times the value measured on GB300 over the full
workload of that process (the whole batch, or its first events where the
oracle covers only those): median, 99th percentile and maximum of the
per-event relative error.  A regression of the FP32 amplitudes or of the
hi/lo split by an order of magnitude fails them; the paper's own check of its
mixed mode (Sect. 3) is agreement within about 1e-5."""

# process -> (median, p99, max)
MIXED_BOUNDS = {
    "e+ e- > mu+ mu-": (2e-6, 5e-6, 1e-5),    # measured 1.2e-7 / 4.3e-7 / 6.6e-7
    "g g > t t~": (2e-6, 6e-6, 1e-5),         # measured 1.8e-7 / 5.3e-7 / 8.8e-7
    "g g > t t~ g": (3e-6, 1e-5, 1e-4),       # test-only process, no full workload: between gg->tt~ and gg->tt~gg
    "g g > t t~ g g": (3e-6, 1e-5, 3e-4),     # measured 3.0e-7 / 9.3e-7 / 3.1e-5
    "g g > t t~ g g g": (6e-6, 2e-5, 1e-3),   # measured 5.5e-7 / 1.3e-6 / 1.1e-4
    "u u~ > t t~": (2e-6, 5e-6, 1e-5),        # measured 1.4e-7 / 4.7e-7 / 8.2e-7
    "u u~ > t t~ g": (2e-6, 6e-6, 3e-5),      # measured 1.4e-7 / 5.5e-7 / 2.4e-6
    "u u~ > t t~ g g": (3e-6, 1e-5, 3e-4),    # not yet measured on a full workload: the gg -> t t~ g g bounds
}


def check_mixed(proc, rel):
    """Assert the median, p99 and max of per-event relative errors rel."""
    import numpy as np
    med, p99, mx = MIXED_BOUNDS[proc]
    assert np.median(rel) <= med, f"{proc}: median {np.median(rel):.3e} > {med:g}"
    assert np.quantile(rel, 0.99) <= p99, f"{proc}: p99 {np.quantile(rel, 0.99):.3e} > {p99:g}"
    assert rel.max() <= mx, f"{proc}: max {rel.max():.3e} > {mx:g}"
