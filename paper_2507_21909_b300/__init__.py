"""B300-native triad-ATRG coarse-graining step (arXiv 2507.21909).

The compute path is the in-tree CUDA library ``libtrg.so`` (sm_103a); ``_lib`` is a
thin ctypes binding with the same entry-point names as ``include/trg.h``.  Accessing
any entry point fails loudly (ImportError) if the library has not been built with
``python -m paper_2507_21909_b300.build``; there is no CPU fallback.
"""
_NAMES = ("TRG_PREC_BF16X3", "TRG_PREC_BF16X10", "TRG_PREC_OZ4", "TRG_PREC_OZ5", "TRG_PREC_OZ6", "TRG_PREC_TF32X3", "TRG_PREC_OZ7", "TRG_PREC_BF16X6", "TRG_PREC_FP64", "TrgError", "lib",
          "library_path", "trg_diag", "trg_finalize", "trg_free_energy", "trg_get_state",
          "trg_init_clock", "trg_init_ising", "trg_magnetisation_impurity", "trg_set_params",
          "trg_set_state", "trg_set_stream", "trg_step", "EXPORTED", "trg_step_timings",
          "PHASES", "trg_gemm", "trg_kernel_stats", "trg_state_dims", "trg_mem_stats",
          "TRG_SKETCH_IN", "TRG_SKETCH_PARAMS", "trg_sketch_set_net", "trg_sketch_get_net",
          "trg_sketch_forward", "trg_sketch_grad", "trg_sketch_train", "trg_set_sketch_mode",
          "trg_sketch_collect", "trg_sketch_fetch", "trg_sketch_stats", "trg_batch_create",
          "trg_batch_step", "trg_batch_results", "trg_batch_lanes", "trg_batch_free",
          "trg_gu_wen_ratio", "trg_batch_gu_wen", "trg_set_bond_overspan",
          "trg_set_impurity_pair", "trg_internal_energy",
          "trg_atrg_init_ising", "trg_atrg_step", "trg_atrg_free_energy", "trg_atrg_diag",
          "trg_get_scalars", "save_state", "load_state")


def __getattr__(name):
    if name in _NAMES:
        from . import _lib
        return getattr(_lib, name)
    raise AttributeError(name)
