"""GB300-native exact point-to-point shortest paths (BiDS, BiD-A*, Multi-BiDS).

The compute path is the CUDA library ``lib/libppsp.so`` behind the C ABI in
``include/ppsp.h``; :mod:`.ppsp` is its Python binding.  Importing this package
does not load the library; :func:`ppsp.load` does, and raises if it is missing.
"""

__all__ = ["ppsp"]
