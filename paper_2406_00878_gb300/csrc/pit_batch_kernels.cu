// pit_batch_kernels.cu -- one instance of the batched kernel per compilation: the build
// compiles this file once per level-solve precision (PIT_BK_FP32 = 0 or 1) and closure
// (PIT_BK_CLOSURES = 1, 2, 4 or 8: closure_bit(conv, nlv)), so that each kernel holds only
// its closure's wave body (a kernel holding two measured 20-25 % slower per job);
// pit_batch.cu picks one by name.
#include <type_traits>

#include "pit_kernels.cuh"

#if !defined(PIT_BK_FP32) || !defined(PIT_BK_CLOSURES)
#error "compile with -DPIT_BK_FP32=0|1 -DPIT_BK_CLOSURES=1|2|4|8"
#endif
#if PIT_BK_CLOSURES != 1 && PIT_BK_CLOSURES != 2 && PIT_BK_CLOSURES != 4 && PIT_BK_CLOSURES != 8
#error "PIT_BK_CLOSURES must be one closure"
#endif

#define PIT_BK_NAME2(f, c) pit_batch_kernel_##f##_##c
#define PIT_BK_NAME(f, c) PIT_BK_NAME2(f, c)

__attribute__((visibility("hidden"))) const void* PIT_BK_NAME(PIT_BK_FP32, PIT_BK_CLOSURES)() {
    using T = typename std::conditional<PIT_BK_FP32 != 0, float, double>::type;
    return reinterpret_cast<const void*>(pit::batch_kernel<pit::kBatchThreads, T, PIT_BK_CLOSURES>);
}
