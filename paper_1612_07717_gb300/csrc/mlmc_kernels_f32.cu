// mlmc_kernels_f32.cu -- float precision, all kernels, no register cap.
#define MLMC_PREC float
#define MLMC_NS prec_f32
#define MLMC_KNS k_f32
#define MLMC_MINB 1
#define MLMC_ALL 1
#include "mlmc_kernels_inst.inc"
