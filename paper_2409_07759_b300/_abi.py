"""ctypes binding of libswgs (include/swgs.h): structure mirrors and function
prototypes, nothing else. Every computation runs inside the library; this
module only marshals arguments.

Loading fails loudly if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libswgs.so"

(SWGS_OK, SWGS_EINVAL, SWGS_ENOMEM, SWGS_ECUDA, SWGS_ETIMEOUT, SWGS_EDEVICE, SWGS_ESTATE,
 SWGS_EPENDING) = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EDEVICE",
                6: "ESTATE", 7: "EPENDING"}

EXPORT_RECORD_SLOT = 0
EXPORT_RECORD_VIEW = 1
EXPORT_RECORD_TILES = 2
EXPORT_RECORD_DEPTH = 3
EXPORT_RECORD_RECT = 4
EXPORT_SORTED_SLOT = 5
EXPORT_TILE_RANGES = 6
EXPORT_LAST = 7
EXPORT_FINAL_T = 8
EXPORT_GRAD2D = 9
EXPORT_RECORD_2D = 10
EXPORT_VIEW_TABLE = 11

NOALLOC_MAX_SLOTS = 1 << 24   # SWGS_NOALLOC_MAX_SLOTS


class SwgsConfig(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("batch", C.c_int32),
                ("near_plane", C.c_float), ("blocks_per_sm", C.c_int32),
                ("count_pairs", C.c_int32), ("pixels_per_thread", C.c_int32),
                ("bwd_pixels_per_thread", C.c_int32), ("bwd_batch", C.c_int32),
                ("sort_single_pass", C.c_int32), ("deferred_sizing", C.c_int32)]


class SwgsGaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("start", C.c_void_p),
                ("expire", C.c_void_p), ("birth", C.c_void_p), ("frozen", C.c_void_p),
                ("capacity", C.c_int64), ("sh_degree", C.c_int32)]


class SwgsView(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("R", C.c_float * 9), ("t", C.c_float * 3), ("frame", C.c_int32)]


class SwgsSavedInfo(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("n_batches", C.c_int32), ("n_records", C.c_int64),
                ("n_keys", C.c_int64), ("n_tiles", C.c_int64), ("n_pixels", C.c_int64),
                ("pairs", C.c_int64), ("n_sort_keys", C.c_int64), ("n_supers", C.c_int64),
                ("device_bytes", C.c_int64), ("record_bytes", C.c_int64)]


class SwgsSgldParams(C.Structure):
    _fields_ = [("lr_means", C.c_float), ("lr_log_scales", C.c_float), ("lr_quats", C.c_float),
                ("lr_logits", C.c_float), ("lr_sh_dc", C.c_float), ("lr_sh_rest", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("noise_lr", C.c_float), ("noise_k", C.c_float), ("noise_t", C.c_float),
                ("adam", C.c_int32), ("relocate", C.c_int32), ("max_n", C.c_int32),
                ("mean_grad_decay", C.c_float), ("window_start", C.c_int32),
                ("swin_size", C.c_int32), ("clear_grads", C.c_int32)]


class SwgsRegParams(C.Structure):
    _fields_ = [("opacity_reg", C.c_float), ("scale_reg", C.c_float),
                ("n_views_total", C.c_int32)]


class SwgsAdamState(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in
                ("m_means", "v_means", "m_log_scales", "v_log_scales", "m_quats", "v_quats",
                 "m_logits", "v_logits", "m_sh", "v_sh")]


NUM_STAGES = 14
STAGE_NAMES = ["compact", "preprocess", "depth_sort", "key_scan", "emit", "tile_sort", "ranges",
               "blend_fwd", "blend_bwd", "preprocess_bwd", "loss", "sgld", "relocate", "update"]


class SwgsProfile(C.Structure):
    _fields_ = [("ms", C.c_double * NUM_STAGES), ("calls", C.c_int64 * NUM_STAGES)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)

# (name, restype, argtypes) for every entry point declared in include/swgs.h
PROTOTYPES = [
    ("swgs_abi_version", C.c_int32, []),
    ("swgs_default_config", C.c_int, [C.POINTER(SwgsConfig)]),
    ("swgs_create", C.c_int, [C.POINTER(SwgsConfig), ALLOC_FN, FREE_FN, C.c_void_p,
                              C.POINTER(C.c_void_p)]),
    ("swgs_destroy", None, [C.c_void_p]),
    ("swgs_last_error", C.c_char_p, [C.c_void_p]),
    ("swgs_active_ids", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    ("swgs_active_ids_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                          C.c_void_p, C.c_void_p, C.c_void_p]),
    ("swgs_frame_update", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int64, C.c_int64,
                                    C.POINTER(SwgsGaussians), C.c_int32, C.c_void_p]),
    ("swgs_render_fwd", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int32,
                                  C.POINTER(SwgsView), C.POINTER(C.c_float),
                                  C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                  C.POINTER(C.c_void_p), C.c_void_p]),
    ("swgs_render_fwd_rgb8", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int32,
                                       C.POINTER(SwgsView), C.POINTER(C.c_float),
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32,
                                       C.POINTER(C.c_void_p), C.c_void_p]),
    ("swgs_render_fwd_l1", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int32,
                                     C.POINTER(SwgsView), C.POINTER(C.c_float),
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p,
                                     C.c_int32, C.POINTER(C.c_void_p), C.c_void_p]),
    ("swgs_render_fwd_l1_u8", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int32,
                                        C.POINTER(SwgsView), C.POINTER(C.c_float),
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                        C.c_void_p, C.c_int32, C.POINTER(C.c_void_p),
                                        C.c_void_p]),
    ("swgs_render_bwd_reg", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_void_p,
                                      C.POINTER(C.c_void_p), C.POINTER(SwgsGaussians),
                                      C.POINTER(SwgsRegParams), C.c_void_p, C.c_void_p]),
    ("swgs_slice_packet_bytes", C.c_size_t, [C.c_int64, C.c_int64]),
    ("swgs_slice_encode", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int64, C.c_int64,
                                    C.c_void_p, C.c_size_t, C.c_int32, C.POINTER(C.c_size_t),
                                    C.c_void_p]),
    ("swgs_slice_decode", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int32,
                                    C.POINTER(SwgsGaussians), C.c_int64, C.c_void_p]),
    ("swgs_mature", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int64, C.c_int32,
                              C.c_int32, C.POINTER(C.c_int64), C.POINTER(SwgsGaussians),
                              C.c_int32, C.POINTER(C.c_int64), C.c_void_p]),
    ("swgs_schedule_expire", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_int64,
                                       C.c_int32, C.c_void_p]),
    ("swgs_render_bwd", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.c_void_p,
                                  C.POINTER(C.c_void_p), C.POINTER(SwgsGaussians), C.c_void_p]),
    ("swgs_saved_release", C.c_int, [C.c_void_p, C.c_void_p]),
    ("swgs_saved_query", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(SwgsSavedInfo)]),
    ("swgs_saved_status", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    ("swgs_saved_export", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t,
                                    C.c_void_p]),
    ("swgs_saved_count", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    ("swgs_loss_l1", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(SwgsView),
                               C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                               C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]),
    ("swgs_sgld_step", C.c_int, [C.c_void_p, C.POINTER(SwgsGaussians), C.POINTER(SwgsGaussians),
                                 C.POINTER(SwgsAdamState), C.POINTER(C.c_int32), C.c_int32,
                                 C.POINTER(SwgsSgldParams), C.c_uint64, C.c_uint64, C.c_void_p,
                                 C.POINTER(C.c_int64), C.c_void_p]),
    ("swgs_slice_range", C.c_int, [C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]),
    ("swgs_profile_enable", C.c_int, [C.c_void_p, C.c_int32]),
    ("swgs_profile_read", C.c_int, [C.c_void_p, C.POINTER(SwgsProfile), C.c_int32]),
    ("swgs_kernel_launches", C.c_int64, []),
    ("swgs_selftest_sort_timeout", C.c_int, [C.c_void_p, C.c_void_p]),
    ("swgs_grad_pack", C.c_int,
     [C.c_void_p, C.POINTER(SwgsGaussians), C.POINTER(SwgsGaussians), C.POINTER(C.c_int32),
      C.c_int32, C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("swgs_grad_unpack", C.c_int,
     [C.c_void_p, C.POINTER(SwgsGaussians), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("swgs_fp32_peak_launch", C.c_int,
     [C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
]

_lib = None


# The struct layouts above mirror include/swgs.h at this SWGS_ABI_VERSION.
ABI_VERSION = 5


def load():
    """Load libswgs.so (raises if it is missing -- there is no CPU fallback)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"libswgs.so not built ({LIB_PATH}); run "
                               "python -m paper_2409_07759_b300.build")
        lib = C.CDLL(str(LIB_PATH))
        for name, res, args in PROTOTYPES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if lib.swgs_abi_version() != ABI_VERSION:
            raise RuntimeError(f"libswgs.so has ABI version {lib.swgs_abi_version()}, this "
                               f"binding mirrors version {ABI_VERSION}: rebuild the library")
        _lib = lib
    return _lib


class SwgsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"swgs {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
