"""GB300-native particle path of the non-hybrid PDF method (Bakosi, Franzese & Boybeyi).

``Context`` wraps the CUDA library ``libpdfx.so`` (C ABI in ``include/pdfx.h``);
``synth`` builds seeded synthetic grids and fields; ``build`` compiles the library for
sm_103a.  The binding is loaded lazily so that input generation works without a GPU.
"""
from . import synth  # noqa: F401


def __getattr__(name):
    if name in ("Context", "PdfxError", "lib", "make_params", "library_path"):
        from . import _binding
        return getattr(_binding, name)
    raise AttributeError(name)
