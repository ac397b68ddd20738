"""Seeded synthetic inputs for the bidomain time step.

This package holds geometry and configuration only: structured meshes, the
heart/torso element labels, per-element fibre frames, stimulus sites and the
physical parameters of each workload.  It contains none of the method's
arithmetic (no assembly, no ionic model, no solver), so both the CPU oracle and
the CUDA library can take their inputs from it.
"""
from .meshes import (  # noqa: F401
    torso_square_2d,
    slab_3d,
    params_2d,
    params_3d,
    stimulus_left_apex,
    stimulus_seeded_disc,
    stimulus_centre_ball,
    batched_slices,
    Mesh,
)
