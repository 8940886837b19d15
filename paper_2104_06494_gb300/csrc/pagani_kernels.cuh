// The per-family kernel tables: every kernel of one integrand family, per
// dimension, as the host runtime dispatches them.
#pragma once
#include "pagani_grad.cuh"

namespace pg {

template <template <int> class FamOf, int THREADS>
FamilyKernels make_family_kernels() {
  FamilyKernels k = {};
  k.threads = THREADS;
#define PG_SET(NN)                                                                              \
  k.loop[NN] = &launch_loop<FamOf<NN>, NN, THREADS>;                                            \
  k.fill[NN] = &launch_fill<FamOf<NN>, NN>;                                                     \
  k.grad[NN] = &launch_grad<FamOf<NN>, NN>;                                                     \
  k.batch_eval[NN] = &launch_batch_eval<FamOf<NN>, NN, THREADS>;                                \
  k.batch_fill[NN] = &launch_batch_fill<FamOf<NN>, NN>;                                         \
  k.batch_eval_fn[NN] = (const void*)&k_evaluate_batch<FamOf<NN>, NN, THREADS>;                 \
  cudaFuncSetAttribute((const void*)&k_evaluate_batch<FamOf<NN>, NN, THREADS>,                  \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));          \
  k.fill_fn[NN] = (const void*)&k_factor_cache<FamOf<NN>, NN>;                                  \
  k.standalone[NN] = &launch_standalone<FamOf<NN>, NN, THREADS, false>;                         \
  k.standalone_diag[NN] = &launch_standalone<FamOf<NN>, NN, THREADS, true>;                     \
  k.loop_fn[NN] = (const void*)&k_evaluate_loop<FamOf<NN>, NN, THREADS>;                        \
  k.table_bytes_per_thread[NN] = (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN);           \
  cudaFuncSetAttribute((const void*)&k_evaluate_loop<FamOf<NN>, NN, THREADS>,                   \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));          \
  cudaFuncSetAttribute((const void*)&k_evaluate_standalone<FamOf<NN>, NN, THREADS, false>,      \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));          \
  cudaFuncSetAttribute((const void*)&k_evaluate_standalone<FamOf<NN>, NN, THREADS, true>,       \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));
  PG_SET(2) PG_SET(3) PG_SET(4) PG_SET(5) PG_SET(6) PG_SET(7) PG_SET(8)
#undef PG_SET
  return k;
}

// The Genz-Malik degree-7 variant: the loop, factor-cache fill and
// standalone kernels (no batched form, no gradient).
template <template <int> class FamOf, int THREADS>
FamilyKernels make_family_kernels_gm7() {
  FamilyKernels k = {};
  k.threads = THREADS;
#define PG_SET(NN)                                                                              \
  k.loop[NN] = &launch_loop<FamOf<NN>, NN, THREADS, 7>;                                         \
  k.fill[NN] = &launch_fill<FamOf<NN>, NN>;                                                     \
  k.fill_fn[NN] = (const void*)&k_factor_cache<FamOf<NN>, NN>;                                  \
  k.standalone[NN] = &launch_standalone<FamOf<NN>, NN, THREADS, false, 7>;                      \
  k.standalone_diag[NN] = &launch_standalone<FamOf<NN>, NN, THREADS, true, 7>;                  \
  k.loop_fn[NN] = (const void*)&k_evaluate_loop<FamOf<NN>, NN, THREADS, 7>;                     \
  k.table_bytes_per_thread[NN] = (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN);           \
  cudaFuncSetAttribute((const void*)&k_evaluate_loop<FamOf<NN>, NN, THREADS, 7>,                \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));          \
  cudaFuncSetAttribute((const void*)&k_evaluate_standalone<FamOf<NN>, NN, THREADS, false, 7>,   \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));          \
  cudaFuncSetAttribute((const void*)&k_evaluate_standalone<FamOf<NN>, NN, THREADS, true, 7>,    \
                       cudaFuncAttributeMaxDynamicSharedMemorySize,                            \
                       (int)(sizeof(typename FamOf<NN>::T) * kCodes * NN * THREADS));
  PG_SET(2) PG_SET(3) PG_SET(4) PG_SET(5) PG_SET(6) PG_SET(7) PG_SET(8)
#undef PG_SET
  return k;
}

template <class F>
struct Fixed {
  template <int N>
  using type = F;
};

}  // namespace pg
