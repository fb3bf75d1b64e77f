"""GB300 (sm_103a) removal-effect rasterizer of POTR (arXiv 2601.14821) and its consumers.

The compute path is ``libpotr.so`` (hand-written CUDA, C ABI in ``include/potr.h``); this
package is its ctypes binding (``_binding``: same names as the C entry points) and the drivers
that own the torch device buffers:

* ``pipeline``  -- ``RemovalEffectFrame`` (preprocess -> bin_sort -> render / removal effect /
  backward on one frame of views) and ``HostPipeline`` (steps fed from pinned host memory);
* ``batched``   -- view chunks sharing a buffer pool, CUDA-graph capture, the autotuner;
* ``autograd``  -- ``torch.autograd.Function`` over render / render_backward;
* ``prune``     -- the iterative pruning controller (Section IV-C);
* ``sh_compact``-- SH energy compaction (Section IV-D);
* ``codec``     -- encoder and decoder of the bitstream (Section IV-E);
* ``finetune``  -- the fine-tuning loop and the POTR-FT cycle (Section IV-F);
* ``compress``  -- the four chained: pruning, SH compaction, encoding (or POTR-FT) in one call;
* ``dist``      -- one process per GPU, ordered cross-rank sums.

Build with ``build.build()``; there is no CPU fallback.
"""
from ._binding import (  # noqa: F401
    POTR_ERR_CAPACITY,
    POTR_ERR_CORRUPT,
    POTR_ERR_CUDA,
    POTR_ERR_INVALID_ARGUMENT,
    POTR_ERR_NUMERIC,
    POTR_ERR_TIMEOUT,
    POTR_ERR_TOO_LARGE,
    POTR_ERR_UNSUPPORTED,
    POTR_OK,
    PotrError,
    lib,
    make_config,
    potr_adam_schedule,
    potr_adam_step,
    potr_adam_step_scheduled,
    potr_bin_sort,
    potr_bin_sort_static,
    potr_bin_sort_workspace_size,
    potr_codec_decode,
    potr_codec_encode,
    potr_preprocess,
    potr_prune_apply,
    potr_prune_select,
    potr_removal_effect,
    potr_render,
    potr_render_backward,
    potr_sh_compact,
    potr_view_layout,
    status_string,
)
