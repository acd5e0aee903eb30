"""Seeded synthetic row-column-array (RCA) workloads.

This package is the one input source shared by the FP64 oracle (``oracle/``)
and the CUDA library (``paper_2511_21647_gb300``).  It holds the acquisition
model that *produces* channel data (scatterers, pulse, noise) and none of the
beamforming / localisation arithmetic of the method; neither side imports the
other, both import this.
"""
from .rca_sim import (  # noqa: F401
    RcaGeometry,
    RcaWorkload,
    WORKLOADS,
    workload,
    batch_workloads,
    scatterer_fields,
    synth_rf,
    generate,
    quantize_int16,
    tx_angles,
)
from .track_scene import TrackScene, track_scene  # noqa: F401,E402
from .slice_scene import moving_slices  # noqa: F401,E402
