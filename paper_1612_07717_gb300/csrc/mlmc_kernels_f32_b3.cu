// mlmc_kernels_f32_b3.cu -- float precision, persistent kernels with 3 resident blocks per SM (<= 85 registers).
#define MLMC_PREC float
#define MLMC_NS prec_f32_b3
#define MLMC_KNS k_f32_b3
#define MLMC_MINB 3
#define MLMC_ALL 0
#include "mlmc_kernels_inst.inc"
