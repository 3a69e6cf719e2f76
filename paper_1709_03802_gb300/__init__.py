"""GB300 (sm_103a) ray-propagation sweep of DART-Ray V2 (Natale et al. 2017).

The computation lives in libdartray.so (include/dartray.h); this package holds
its CUDA sources (csrc/), the build step and a thin ctypes binding.
"""
from .dartray import (DartRay, DartRayBatch, DartRayError, dust_self_heating, external_map, rfed_albedo, default_params, load, library_path, EXPORTED,
                      dartray_params_default, dartray_grid_create, dartray_direct, dartray_scatter_iter,
                      dartray_rfed, dartray_jsca_layout, dartray_jsca, dartray_map, dartray_map_noalloc, dartray_state_save,
                      dartray_state_load, dartray_grid_destroy)

__all__ = ["DartRay", "DartRayBatch", "DartRayError", "dust_self_heating", "external_map", "rfed_albedo", "default_params", "load", "library_path", "EXPORTED",
           "dartray_params_default", "dartray_grid_create", "dartray_direct", "dartray_scatter_iter",
           "dartray_rfed", "dartray_jsca_layout", "dartray_jsca", "dartray_map", "dartray_map_noalloc", "dartray_state_save",
           "dartray_state_load", "dartray_grid_destroy"]
