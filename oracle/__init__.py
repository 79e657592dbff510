"""FP64 CPU oracle for the near-field (P2P) operator -- test infrastructure.

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
package.  The CUDA library never imports, links or calls it, and it shares no
code with the library.  See ``p2p_oracle.c`` for the definitions it follows.
"""
from .oracle import (  # noqa: F401
    build, load, num_threads, set_num_threads, morton, unmorton, cells, tree, redundant, Context,
    gravity, helmholtz, pair_count, helmholtz_adjoint, gravity_adjoint,
)
