"""Seeded synthetic inputs for the BDDC Darcy solver and its CPU oracle.

This package is shared by the oracle (``oracle/``) and by the GPU library's
tests and benchmark.  It only produces *inputs*: grids, permeability fields,
subdomain partitions and forcing (sources, boundary conditions).  It contains
none of the method's arithmetic (no discretisation, no solver).

The fields stand in for the SPE10 model-2 permeability data (Sec. 5), which is
not available: they reproduce its grid shape (60 x 220 x 85 cells of
20 x 10 x 2 ft), its high contrast (six or more orders of magnitude) and the
structure of its two halves (smooth upper layers, fluvial channels below).
"""

from .problems import (  # noqa: F401
    Grid,
    Problem,
    box_partition,
    irregular_box_partition,
    lognormal_iid,
    gaussian_field,
    channelized_2d,
    layered_3d,
    pressure_drop_bc,
    directional_pressure_bc,
    no_flow_bc,
    corner_wells,
    make_config,
    n_faces,
    face_axis_counts,
)
