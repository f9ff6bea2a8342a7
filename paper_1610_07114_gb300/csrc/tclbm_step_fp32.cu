// Step kernels with fp32 population storage.
#include "tclbm_device.cuh"
namespace tclbm {
using ST = float;
}
#define LAUNCH_FN launch_step_fp32
#define PREPARE_FN prepare_step_fp32
#define BATCH_FN launch_batch_fp32
#define BATCH_OCC_FN batch_occupancy_fp32
#define BATCH_TMA_FN launch_batch_tma_fp32
#define TMA_RESIDENT_FN tma_resident_fp32
#include "tclbm_step_inst.cuh"
