"""GB300 (sm_103a) library for the affine reconstructed nodal DG method (arXiv 1912.06221):
the convection-diffusion right-hand side with parallelogram reconstruction on every edge,
fused SSP-RK3 stepping and CUDA-graph replay, behind the C ABI in include/rdg.h."""
from .rdg import (Solver, Batch, load, query_bytes, reference_operator, peak_fma, stream_read_seconds, RdgError, BC_PERIODIC, BC_DIRICHLET,
                  FP32, FP64, FP32_3XTF32, TAU_CONST, TAU_COS, TAU_SIN, IFACE_ALG2, IFACE_HARMONIC, IFACE_ALG1, SSP_RK3, LSRK54, np_of,
                  STAGE_AUTO, STAGE_TWO_KERNELS, STAGE_ONE_KERNEL, BATCH_AUTO, BATCH_GRAPH, BATCH_PERSISTENT)

__all__ = ["Solver", "Batch", "load", "query_bytes", "reference_operator", "peak_fma", "stream_read_seconds", "RdgError", "BC_PERIODIC", "BC_DIRICHLET",
           "FP32", "FP64", "FP32_3XTF32", "TAU_CONST", "TAU_COS", "TAU_SIN", "IFACE_ALG2", "IFACE_HARMONIC", "IFACE_ALG1", "SSP_RK3", "LSRK54", "np_of",
           "STAGE_AUTO", "STAGE_TWO_KERNELS", "STAGE_ONE_KERNEL", "BATCH_AUTO", "BATCH_GRAPH", "BATCH_PERSISTENT"]
