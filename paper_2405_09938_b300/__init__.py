"""B300-native bistatic SAR/ATI facet-to-IQ echo generator.

The compute path is ``libharm.so`` (hand-written CUDA for sm_103a behind the C ABI
in ``include/harm.h``); :mod:`paper_2405_09938_b300.harm` is its ctypes binding.
"""
from .harm import (HARM_C64, HARM_C128, HARM_PREC_FP64, HARM_PREC_MIXED, HarmError, Scene,
                   harm_echo_accumulate, harm_echo_adjoint, harm_facets_generate, harm_last_error,
                   harm_scene_create, harm_scene_destroy, harm_scene_query, harm_scene_set_cells,
                   harm_scene_sync, load_library)

__all__ = [
    "HARM_C64", "HARM_C128", "HARM_PREC_FP64", "HARM_PREC_MIXED", "HarmError", "Scene",
    "harm_echo_accumulate", "harm_echo_adjoint", "harm_facets_generate", "harm_last_error",
    "harm_scene_create", "harm_scene_destroy", "harm_scene_query", "harm_scene_set_cells",
    "harm_scene_sync", "load_library",
]
