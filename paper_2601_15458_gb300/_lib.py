"""ctypes binding of libmsa.so (argument marshalling only).

The library is built in-tree by :func:`paper_2601_15458_gb300.build.build`.
If it is missing, every call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "libmsa.so")

_lib = None
_lock = threading.Lock()

c_void_p, c_int32, c_int64, c_float = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float

MSA_OK, MSA_EINVAL, MSA_ENOMEM, MSA_ECUDA, MSA_ETIMEOUT, MSA_EUNSUPPORTED, MSA_EDATA = range(7)
MSA_DNA, MSA_PROTEIN = 0, 1


class SeqSetC(ctypes.Structure):
    _fields_ = [("ascii", c_void_p), ("offs", c_void_p), ("codes", c_void_p), ("planes", c_void_p),
                ("total", c_int64), ("n_seqs", c_int32), ("alphabet", c_int32), ("max_len", c_int32),
                ("reserved", c_int32)]


# name -> (restype, argtypes); the declarations of include/msa.h
SIGNATURES = {
    "msa_ctx_create": (c_int32, [ctypes.POINTER(c_void_p), c_int32, c_int64]),
    "msa_ctx_destroy": (None, [c_void_p]),
    "msa_ctx_check": (c_int32, [c_void_p, c_void_p]),
    "msa_last_error": (ctypes.c_char_p, [c_void_p]),
    "msa_version": (ctypes.c_char_p, []),
    "msa_prof_enable": (c_int32, [c_void_p, c_int32]),
    "msa_prof_read": (c_int32, [c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_int64), c_int32]),
    "msa_code_bytes": (c_int64, [c_int64]),
    "msa_plane_words": (c_int64, [c_int64, c_int32]),
    "msa_lev_workspace_bytes": (c_int64, [c_int64, c_int32]),
    "msa_pack": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p]),
    "msa_lev_batch": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_int64, c_void_p, c_void_p]),
    "msa_lev_autotune": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_int64, c_void_p, c_void_p]),
    "msa_lev_batch_noalloc": (c_int32, [ctypes.POINTER(SeqSetC), c_void_p, c_int64, c_void_p, c_void_p]),
    "msa_nw_align_batch": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32, c_void_p, c_int64,
                                     c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "msa_nw_workspace_bytes": (c_int64, [c_int32, c_int32]),
    "msa_nw_align_batch_affine": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32, c_void_p,
                                            c_int64, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p]),
    "msa_lev_banded_batch": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_int64, c_void_p, c_void_p,
                                       c_void_p, c_void_p]),
    "msa_lev_banded_workspace_bytes": (c_int64, [c_int64, c_int32]),
    "msa_mlp_num_params": (c_int32, []),
    "msa_mlp_state_bytes": (c_int64, []),
    "msa_mlp_sync": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "msa_kmer_profile": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p]),
    "msa_pair_features": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_int64, c_void_p,
                                    c_void_p]),
    "msa_mlp_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "msa_mlp_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_int32, c_float,
                                     c_float, c_void_p, c_void_p]),
    "msa_mlp_train_workspace_bytes": (c_int64, [c_int32]),
    "msa_mlp_read_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "msa_band_predict": (c_int32, [c_void_p, c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_int64,
                                   c_float, c_int32, c_void_p, c_void_p, c_void_p]),
    "msa_lev_one_to_many": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_int32, c_void_p, c_int64, c_void_p,
                                      c_void_p]),
    "msa_lev_one_to_many_workspace_bytes": (c_int64, [c_int64, c_int32]),
    "msa_lev_tune_get": (c_int32, [c_void_p, c_void_p]),
    "msa_lev_tune_set": (c_int32, [c_void_p, c_void_p]),
    "msa_band_calibrate": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_void_p]),
    "msa_clam_partition": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "msa_clam_partition_banded": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_float, c_int32,
                                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p]),
    "msa_merge_tree": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_void_p, c_void_p,
                                 c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                 c_void_p, c_void_p]),
    "msa_merge_tree_affine": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p,
                                        c_void_p, c_void_p, c_void_p]),
    "msa_msa_metrics": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_int32, c_int32, c_void_p, c_void_p,
                                  c_int32, ctypes.c_uint8, c_void_p, c_void_p, c_void_p]),
    "msa_msa_rows": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_int32, c_void_p,
                               c_void_p]),
    "msa_probe_int_pipe": (c_int32, [c_void_p, c_int32, c_int32, ctypes.POINTER(c_int64), c_void_p]),
    "msa_nw_align_batch_affine_sub": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32, c_void_p,
                                                c_int64, c_void_p, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                                c_void_p, c_void_p, c_void_p]),
    "msa_nw_align_batch_anchored": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32, c_void_p,
                                              c_int64, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                              c_void_p, c_void_p, c_void_p]),
    "msa_nw_align_batch_anchored_affine": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32,
                                                     c_void_p, c_int64, c_int32, c_int32, c_int32, c_int32, c_int32,
                                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "msa_nw_align_batch_anchored_affine_sub": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_int64, c_int32,
                                                         c_void_p, c_int64, c_int32, c_void_p, c_int32, c_int32,
                                                         c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "msa_merge_tree_affine_sub": (c_int32, [c_void_p, ctypes.POINTER(SeqSetC), c_void_p, c_void_p, c_void_p,
                                            c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_int32, c_int32,
                                            c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
}


def lib():
    """The loaded library; raises RuntimeError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO_PATH):
                raise RuntimeError(f"{SO_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(SO_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols():
    return list(SIGNATURES)
