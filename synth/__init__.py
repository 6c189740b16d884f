"""Seeded synthetic photoacoustic RF frames and the workload table.

This package is shared by the oracle tests, the GPU parity tests and
``bench.py`` as a source of *input data only*.  It simulates the forward
problem (point and line absorbers radiating an N-shaped pulse that reaches
each element after the one-way time of flight) and holds none of the
beamformer's arithmetic: no delay tables, interpolation, roots, power sums,
filtering or envelope detection live here.

The paper's own data (k-Wave simulations, the ex-vivo chicken-breast scan,
Sections 3 and 4) is not available; these frames stand in for it with the
shapes, sample rates and target structures of the five workload
configurations listed in :mod:`synth.configs`.
"""

from .configs import CONFIGS, workload, serving_mix  # noqa: F401
from .rf import (  # noqa: F401
    Scene,
    point_scene,
    make_scene,
    render_rf,
    make_frame,
    make_frames,
    quantize,
)
