// Executor instantiation: FP32 storage, tensor-core (tcgen05) updates (the split-bf16 / bf16 / fp16 precisions).
#include "executor.cuh"

namespace tqr {

int exec_launch_mixed(const ExecParams &p, void *stream, size_t smem) {
  return launch_typed<float, float, true>(p, stream, smem);
}

int exec_slots_mixed(size_t smem) { return slots_typed<float, float, true>(smem); }

}  // namespace tqr
