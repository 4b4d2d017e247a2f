"""GB300-native matrix-free spin-1/2 Heisenberg H.x (XDiag's hot path).

The compute path is the CUDA library ``libxdgpu.so`` (built from ``csrc/``)
reached through ``_lib`` (ctypes, argument marshalling only).  Importing this
package does not load the library; ``api`` does, and raises if it is
missing.  ``workloads`` holds the seeded synthetic inputs.
"""
__all__ = ["workloads"]
