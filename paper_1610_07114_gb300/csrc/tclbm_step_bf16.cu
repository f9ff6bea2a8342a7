// Step kernels with bf16 population storage.
#include "tclbm_device.cuh"
namespace tclbm {
using ST = __nv_bfloat16;
}
#define LAUNCH_FN launch_step_bf16
#define PREPARE_FN prepare_step_bf16
#define BATCH_FN launch_batch_bf16
#define BATCH_OCC_FN batch_occupancy_bf16
#define BATCH_TMA_FN launch_batch_tma_bf16
#define TMA_RESIDENT_FN tma_resident_bf16
#include "tclbm_step_inst.cuh"
