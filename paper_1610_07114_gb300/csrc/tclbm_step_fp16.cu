// Step kernels with fp16 population storage.
#include "tclbm_device.cuh"
namespace tclbm {
using ST = __half;
}
#define LAUNCH_FN launch_step_fp16
#define PREPARE_FN prepare_step_fp16
#define BATCH_FN launch_batch_fp16
#define BATCH_OCC_FN batch_occupancy_fp16
#define BATCH_TMA_FN launch_batch_tma_fp16
#define TMA_RESIDENT_FN tma_resident_fp16
#include "tclbm_step_inst.cuh"
