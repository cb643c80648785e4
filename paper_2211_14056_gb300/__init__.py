"""GB300-native event-parallel MadFlow hot path (arXiv:2211.14056).

The compute path is the CUDA library ``lib/libmadflow_gb300.so`` behind the C
ABI in ``include/madflow_gb300.h``; ``binding`` marshals arguments to it with
ctypes (PyTorch tensors supply device memory and streams).  There is no CPU
fallback: importing the binding without the built library raises.
"""
from .binding import (  # noqa: F401
    MF_ERR_ARG, MF_ERR_CUDA, MF_ERR_UNSUPPORTED, MF_FP32, MF_FP32_TC, MF_FP64, MF_OK, MF_PROC_EE_MUMU,
    MF_PROC_GG_TTX, MF_PROC_GG_TTXG, MF_PROC_GG_TTXGG, MF_PROC_GUX_TTXGUX, MF_PROC_GU_TTXGU, MF_PROC_UG_TTXGU,
    MF_PROC_UUX_TTXGG, MF_PROC_UXG_TTXGUX, MF_PROC_UXU_TTXGG, MF_WARN_CAPACITY, MF_WARN_NEWTON,
    Grid, MFError, Mixed, PDFSet, Process, fma_throughput, kernel_launches, library_path, load_library, uniforms,
)
