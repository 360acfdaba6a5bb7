"""GB300-native exact point-to-point shortest paths: BiDS, BiD-A*, ET and A*
searches, Multi-BiDS and SSSP-based batches, on undirected and directed graphs.

The compute path is the CUDA library ``lib/libppsp.so`` behind the C ABI in
``include/ppsp.h``; :mod:`.ppsp` is its Python binding.  Importing this package
does not load the library; :func:`ppsp.load` does, and raises if it is missing.
Around it: :mod:`.learned_delta` (stepping-increment model), :mod:`.serving`
(continuous batching), :mod:`.autotune` (launch options), :mod:`.replicas`
(query-parallel multi-GPU helpers).
"""

__all__ = ["ppsp"]
