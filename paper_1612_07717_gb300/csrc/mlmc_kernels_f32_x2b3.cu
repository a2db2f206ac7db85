// mlmc_kernels_f32_x2b3.cu -- float precision, persistent kernels with two path pairs per thread on the packed FP32 pipe, 3 resident blocks per SM (<= 85 registers).
#define MLMC_PREC float
#define MLMC_NS prec_f32_x2b3
#define MLMC_KNS k_f32_x2b3
#define MLMC_MINB 3
#define MLMC_ALL 0
#define MLMC_X2 1
#include "mlmc_kernels_inst.inc"
