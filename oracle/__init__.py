"""FP64 CPU oracle of the elastic-wall D3Q19 LBGK step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import it.  The product
package (``paper_2108_08783_gb300``) never does, and the two share no code.
"""
from .oracle import Oracle, velocity_set, equilibrium, collide, bessel_j01, womersley_shape  # noqa: F401
