// Executor instantiation: FP64 storage and arithmetic (the plain FP64 factorization and its apply-Q).
#include "executor.cuh"

namespace tqr {

int exec_launch_f64(const ExecParams &p, void *stream, size_t smem) {
  return launch_typed<double, double, false>(p, stream, smem);
}

int exec_slots_f64(size_t smem) { return slots_typed<double, double, false>(smem); }

}  // namespace tqr
