"""GB300 (sm_103a) removal-effect rasterizer of POTR (arXiv 2601.14821).

The compute path is ``libpotr.so`` (hand-written CUDA, C ABI in ``include/potr.h``); this
package is its ctypes binding (``_binding``: same names as the C entry points) and a frame
driver that owns the torch device buffers (``pipeline``).  Build with ``build.build()``.
"""
from ._binding import (  # noqa: F401
    POTR_ERR_CAPACITY,
    POTR_ERR_CUDA,
    POTR_ERR_INVALID_ARGUMENT,
    POTR_ERR_NUMERIC,
    POTR_ERR_TIMEOUT,
    POTR_ERR_UNSUPPORTED,
    POTR_OK,
    PotrError,
    lib,
    make_config,
    potr_bin_sort,
    potr_bin_sort_workspace_size,
    potr_preprocess,
    potr_removal_effect,
    potr_render,
    potr_view_layout,
    status_string,
)
