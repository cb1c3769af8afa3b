"""GB300-native rasterizer for 3D Student Splatting and Scooping (SSS).

The hot path (projection, binning, sorting, forward and backward compositing,
the SGHMC/Adam step) is CUDA for sm_103a in libsss (include/sss.h); this
package is its thin Python side:

    _abi      ctypes binding with the C names (argument marshalling only)
    frame     device scenes, frames and sampler state on top of the ABI
    inputs    seeded synthetic scenes and cameras (no rasterizer arithmetic)
    build     compiles libsss.so for sm_103a

Importing the package does not load CUDA; the binding loads libsss on first
use and raises if it has not been built (there is no CPU fallback).
"""

__all__ = ["inputs", "build"]
