"""Seeded synthetic inputs for the TPMC hot path: meshes and workloads.

Shared by the oracle-side tests and the CUDA-side tests and benchmark.  This
package holds none of the method's arithmetic (no sampling, no fluxes, no
ray tracing): only geometry and run parameters.
"""
from . import meshes, workloads  # noqa: F401
