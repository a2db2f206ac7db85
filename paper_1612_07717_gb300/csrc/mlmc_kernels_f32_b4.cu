// mlmc_kernels_f32_b4.cu -- float precision, persistent kernels with 4 resident blocks per SM (<= 64 registers).
#define MLMC_PREC float
#define MLMC_NS prec_f32_b4
#define MLMC_KNS k_f32_b4
#define MLMC_MINB 4
#define MLMC_ALL 0
#include "mlmc_kernels_inst.inc"
