// pit_check.cuh -- the bounds-checking build of the level-chain kernels.
//
// Compiled with -DPIT_CHECK_BOUNDS (build.py's check_bounds build, libpit_check.so), the
// arrays of the residual, assembly, level-chain and wavefront kernels are held as Chk<T>:
// a pointer with the index range it may touch and a small id naming the array. Every
// indexed access checks the index; an access outside the range is skipped (a load reads a
// scratch word, a store writes it), the array's id is recorded in a status word of the
// translation unit, and the kernel runs on, so the check never traps, faults or hangs.
// The host reads the word after each synchronising call (pit_bounds_status) and turns a
// recorded id into PIT_EBOUNDS. Without PIT_CHECK_BOUNDS the same code compiles to plain
// pointers (sptr<T> is T*, chk() returns its argument) and the checks vanish.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

namespace pit {

// Ids of the checked arrays (recorded on the first failing access).
enum : int {
    kChkU = 1, kChkU0, kChkBc, kChkQ, kChkR, kChkCoef, kChkDU,         // global problem arrays
    kChkSmem = 16,                                                      // + Smem member index
    kChkUprev = 40, kChkUstrip, kChkDeep, kChkRed,                      // other shared arrays
    kChkPrefix = 50, kChkCellIters, kChkSumsq, kChkProg, kChkTpub,      // wavefront workspace
    kChkPub, kChkFlags, kChkRedPart, kChkLevel,                         // chain workspace
    kChkBulk = 60,                                                      // bulk-copy ranges
};

#ifdef PIT_CHECK_BOUNDS

// First failing array id of this translation unit's kernels (0 = none), and the word
// a skipped access reads or writes.
static __device__ int g_pit_bounds;
static __device__ __align__(16) double g_pit_sink[2];

__device__ __forceinline__ void bounds_fail(int id) { atomicCAS(&g_pit_bounds, 0, id); }

template <typename T>
struct Chk {
    T* p;
    long long lo, hi;  // valid indices i (relative to p): lo <= i < hi
    int id;
    __device__ __forceinline__ T& operator[](long long i) const {
        if (i < lo || i >= hi || p == nullptr) {
            bounds_fail(id);
            return *reinterpret_cast<T*>(g_pit_sink);
        }
        return p[i];
    }
    __device__ __forceinline__ Chk operator+(long long d) const { return Chk{p + d, lo - d, hi - d, id}; }
    __device__ __forceinline__ Chk operator-(long long d) const { return Chk{p - d, lo + d, hi + d, id}; }
    // The range [off, off + len) as an array of its own (checked against this one).
    __device__ __forceinline__ Chk sub(long long off, long long len) const {
        if (off < lo || off + len > hi) bounds_fail(id);
        return Chk{p + off, 0, len, id};
    }
    __device__ __forceinline__ operator T*() const { return p; }  // unchecked: bulk copies, tests for NULL
    // a read-only view of the same range
    template <typename U, typename = typename std::enable_if<std::is_same<U, T>::value && !std::is_const<T>::value>::type>
    __device__ __forceinline__ operator Chk<const U>() const {
        return Chk<const U>{p, lo, hi, id};
    }
};

template <typename T>
using sptr = Chk<T>;

template <typename T>
__device__ __forceinline__ Chk<T> chk(T* p, long long n, int id) {
    return Chk<T>{p, 0, p ? n : 0, id};
}
template <typename T>
__device__ __forceinline__ Chk<T> chk(const Chk<T>& c, long long, int) {
    return c;
}

// Checked cache-global accesses.
__device__ __forceinline__ double ldcg(const Chk<const double>& c) {
    if (c.lo > 0 || c.hi <= 0 || c.p == nullptr) {
        bounds_fail(c.id);
        return 0.0;
    }
    return __ldcg(c.p);
}
__device__ __forceinline__ double ldcg(const Chk<double>& c) {
    return ldcg(Chk<const double>{c.p, c.lo, c.hi, c.id});
}
__device__ __forceinline__ void stcg(const Chk<double>& c, double v) {
    if (c.lo > 0 || c.hi <= 0 || c.p == nullptr) {
        bounds_fail(c.id);
        return;
    }
    __stcg(c.p, v);
}

#define PIT_CHECK(cond, id)                          \
    do {                                             \
        if (!(cond)) ::pit::bounds_fail((id));       \
    } while (0)

// Every translation unit has its own record; each registers a reader with the library at
// load time (no CUDA call there), and pit_bounds_status asks them all.
void register_bounds_reader(int (*reader)());

namespace {
// The first recorded id (cleared), 0 for none, -1 when the device could not be read.
int read_and_clear_bounds() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_pit_bounds, sizeof v) != cudaSuccess) return -1;
    if (v != 0) {
        const int zero = 0;
        if (cudaMemcpyToSymbol(g_pit_bounds, &zero, sizeof zero) != cudaSuccess) return -1;
    }
    return v;
}
struct BoundsReaderRegistration {
    BoundsReaderRegistration() { register_bounds_reader(&read_and_clear_bounds); }
};
BoundsReaderRegistration g_bounds_reader_registration;
}  // namespace

#else

template <typename T>
using sptr = T*;

template <typename T>
__device__ __forceinline__ T* chk(T* p, long long, int) {
    return p;
}
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(double* p, double v) { __stcg(p, v); }

#define PIT_CHECK(cond, id) \
    do {                    \
    } while (0)

#endif

}  // namespace pit
