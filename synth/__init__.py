"""Seeded synthetic inputs for the FS2D HLF problem.

This package is the only code shared by the oracle and the CUDA path. It draws
graphs, diagonals, enumeration windows and index samples from numpy's PCG64 and
holds none of the method's arithmetic (no elimination, no kernel, no q, no
enumeration). Matrices are returned dense (one uint8 per entry); each side packs
them in its own way.
"""

from .grid import (  # noqa: F401
    all_connected,
    b_from_string,
    batch_instances,
    grid_edges,
    grid_instance,
    paper_b_patterns,
    poisson_stream,
    random_regular,
    random_symmetric,
    sample_indices,
    window_offset,
)
