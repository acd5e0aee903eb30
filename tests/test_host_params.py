"""Host-side parameter logic shared by the library's Python binding and the
oracle, checked without a GPU: the decisions both sides take in double
precision (band edges, bin-to-subset assignment inputs, tracking thresholds)
start from bit-identical numbers, and the parameter structs have the
header's layout."""
import ctypes

import numpy as np

from oracle import separation as OSep


def test_default_band_edges_are_bit_identical():
    from paper_2511_21647_gb300 import rca
    for prf in (400.0, 333.0, 1000.0):
        for nb in (1, 2, 3, 4):
            p = rca.make_sep_params(prf, nb)
            got = np.array(p.edges_hz[:nb + 1])
            assert np.array_equal(got, OSep.default_edges(prf, nb)), (prf, nb)
            assert p.n_bands == nb and p.prf_hz == prf


def test_explicit_band_edges_pass_through():
    from paper_2511_21647_gb300 import rca
    edges = [5.0, 30.0, 90.0, 200.0]
    p = rca.make_sep_params(400.0, 3, edges)
    assert list(p.edges_hz[:4]) == edges
    try:
        rca.make_sep_params(400.0, 3, edges[:3])
    except ValueError:
        pass
    else:
        raise AssertionError("a wrong edge count must be rejected")


def test_tracking_thresholds_match_the_oracle():
    import oracle as O
    from paper_2511_21647_gb300 import rca
    g = rca.make_track_params()
    o = O.track_params()
    assert (g.len, g.substeps) == (o.len, o.substeps)
    assert g.max_step_m == o.max_step and g.cos_max_turn == o.cos_max_turn
    assert g.max_speed_change == o.max_speed_change and g.voxel_m == o.voxel


def test_parameter_struct_layouts():
    from paper_2511_21647_gb300 import _lib
    assert ctypes.sizeof(_lib.ulm_sep_params) == 8 + 4 + 4 + 8 * (_lib.ULM_SEP_MAX_BANDS + 1)
    assert _lib.ulm_sep_params.edges_hz.offset == 16
    assert ctypes.sizeof(_lib.ulm_track_params) == 4 + 4 + 4 * 8
