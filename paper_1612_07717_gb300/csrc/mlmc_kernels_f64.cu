// mlmc_kernels_f64.cu -- double precision, all kernels.
#define MLMC_PREC double
#define MLMC_NS prec_f64
#define MLMC_KNS k_f64
#define MLMC_MINB 1
#define MLMC_ALL 1
#include "mlmc_kernels_inst.inc"
