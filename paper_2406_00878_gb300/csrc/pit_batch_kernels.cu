// pit_batch_kernels.cu -- one instance of the batched kernel per compilation: the build
// compiles this file once per level-solve precision (PIT_BK_FP32 = 0 or 1) and closure
// set (PIT_BK_CLOSURES = 1..15, bits closure_bit(conv, nlv)), so that every set gets a
// kernel holding only its closures' wave bodies; pit_batch.cu picks one by name.
#include <type_traits>

#include "pit_kernels.cuh"

#if !defined(PIT_BK_FP32) || !defined(PIT_BK_CLOSURES)
#error "compile with -DPIT_BK_FP32=0|1 -DPIT_BK_CLOSURES=1..15"
#endif
#if PIT_BK_CLOSURES < 1 || PIT_BK_CLOSURES > 15
#error "PIT_BK_CLOSURES must be a non-empty set of the four closures"
#endif

#define PIT_BK_NAME2(f, c) pit_batch_kernel_##f##_##c
#define PIT_BK_NAME(f, c) PIT_BK_NAME2(f, c)

__attribute__((visibility("hidden"))) const void* PIT_BK_NAME(PIT_BK_FP32, PIT_BK_CLOSURES)() {
    using T = typename std::conditional<PIT_BK_FP32 != 0, float, double>::type;
    return reinterpret_cast<const void*>(pit::batch_kernel<pit::kBatchThreads, T, PIT_BK_CLOSURES>);
}
