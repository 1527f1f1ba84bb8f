// Executor instantiation: FP32 storage with SIMT updates (TQR_FP32, the batched FP32 factorization).
#include "executor.cuh"

namespace tqr {

int exec_launch_f32(const ExecParams &p, void *stream, size_t smem) {
  return launch_typed<float, float, false>(p, stream, smem);
}

int exec_slots_f32(size_t smem) { return slots_typed<float, float, false>(smem); }

}  // namespace tqr
