// Host dispatch of the persistent tile-task executor (executor.cuh): shared-memory sizes,
// resident CTAs and the launch of the instantiation a precision needs.  Each
// instantiation is compiled in a translation unit of its own (exec_*.cu) so that the
// build compiles them in parallel.
#include <cuda_runtime.h>

#include <cstdint>

#include "executor.cuh"

namespace tqr {

size_t executor_smem_bytes(int nb, int ib, bool real_is_double, bool apply_q) {
  const size_t ssz = (real_is_double || apply_q) ? sizeof(double) : sizeof(float);
  const size_t bytes = smem_elems(nb, ib, ssz);
  return bytes <= 227 * 1024 ? bytes : 0;
}

size_t mixed_slot_bytes(int nparts) { return slot_bytes(nparts); }

size_t mixed_executor_smem_bytes() { return mixed_smem_bytes(); }

int executor_slots(bool real_is_double, bool mixed, int nb, int ib) {
  if (mixed && !real_is_double) return exec_slots_mixed(mixed_smem_bytes());
  const size_t smem = executor_smem_bytes(nb, ib, real_is_double, false);
  if (real_is_double) return exec_slots_f64(smem);
  return exec_slots_f32(smem);
}

int launch_executor(const ExecParams &p, bool real_is_double, void *stream) {
  if (p.cplx) return zexec_launch(p, stream);
  const bool apply_q = p.B != nullptr;
  if (p.mixed && !apply_q && !real_is_double) return exec_launch_mixed(p, stream, mixed_smem_bytes());
  const size_t smem = executor_smem_bytes(p.nb, p.ib, real_is_double, apply_q);
  if (real_is_double) return exec_launch_f64(p, stream, smem);
  if (apply_q) return exec_launch_f32_apply(p, stream, smem);
  return exec_launch_f32(p, stream, smem);
}

}  // namespace tqr
