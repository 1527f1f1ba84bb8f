// Executor instantiation: FP32 factors applied to an FP64 right-hand side (apply-Q of TQR_FP32 factors).
#include "executor.cuh"

namespace tqr {

int exec_launch_f32_apply(const ExecParams &p, void *stream, size_t smem) {
  return launch_typed<float, double, false>(p, stream, smem);
}

}  // namespace tqr
