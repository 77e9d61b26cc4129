"""GB300-native mixTS-PIMD hot path (arXiv 2411.11988): CUDA library + thin binding."""
from . import analysis  # noqa: F401
from .mixts import (MixTS, MixTSBatch, MixtsError, lib, FP64, FP32_FORCES, LIB_PATH, EXPORTED, THETA_NAMES,  # noqa: F401
                    mixts_potential, alu_peak_tflops)
