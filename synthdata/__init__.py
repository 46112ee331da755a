"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds only random-number plumbing and image synthesis. It holds
none of the inpainting, tonal-optimisation or densification arithmetic, so it
can serve both sides without coupling them.

The images stand in for the paper's twelve 4K nature photographs (Sec. 6.1,
Fig. "dataset"), which are not available: same resolution (3840x2160 RGB),
smooth regions with sharp edges, values on the [0, 255] scale.
"""

from .generators import (  # noqa: F401
    synth_image,
    synth_rgb,
    random_mask,
    batch_specs,
    serving_stream,
    serving_inputs,
)
