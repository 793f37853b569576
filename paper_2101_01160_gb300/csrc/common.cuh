// Shared host/device helpers of libmdlg.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "mdlg.h"

#include <nvtx3/nvToolsExt.h>

namespace mdlg {

// A named NVTX range over the host side of one library call (argument checks
// and the enqueue of its launches), so that a profiler can pick out the
// call's kernels by name (ncu --nvtx --nvtx-include "md_step/").  NVTX is
// header-only; without an attached tool a range is one predictable branch.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
int fail(int code, const char *fmt, ...);

#define MD_CUDA_TRY(expr)                                                         \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess)                                                    \
            return ::mdlg::fail(MD_E_CUDA, "%s:%d %s: %s", __FILE__, __LINE__,     \
                                #expr, cudaGetErrorString(e_));                   \
    } while (0)

// Device status word values (a device-side failure sets one, the host reads
// it at md_sync).
enum DevStatus : int { DS_OK = 0, DS_TIMEOUT = 1, DS_SKIN = 2, DS_NONFINITE = 4, DS_NBR_OVERFLOW = 8, DS_CAPACITY = 16 };

// ---------------------------------------------------------------- device memory order
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acqrel_gpu(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative (co-resident) launch, with a bounded
// wait: a CTA that waits longer than limit_ns sets DS_TIMEOUT in *status and
// leaves the barrier.  Returns false once any failure has been flagged, so
// that every CTA leaves the kernel at its next barrier instead of waiting.
// gen is read once at kernel start into *my_gen (thread 0's copy).
struct GridBarrier {
    unsigned *count;
    unsigned *gen;
    int *status;
};

__device__ __forceinline__ bool grid_sync(const GridBarrier &b, unsigned &my_gen,
                                          uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g = my_gen;
        unsigned old = atom_add_acqrel_gpu(b.count, 1u);
        if (old == gridDim.x - 1) {
            atomicExch(b.count, 0u);
            st_release_gpu(b.gen, g + 1u);
        } else {
            uint64_t t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_gpu(b.gen) == g) {
                if ((++spins & 63u) == 0 && global_ns() - t0 > limit_ns) {
                    atomicOr(b.status, (int)DS_TIMEOUT);
                    break;
                }
                __nanosleep(20);
            }
        }
        my_gen = g + 1u;
        __threadfence();
        s_ok = ((*(volatile int *)b.status) & DS_TIMEOUT) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// Periodic wrap of a cell coordinate that is at most one cell out of range.
__device__ __forceinline__ int wrap1(int c, int n) {
    return c < 0 ? c + n : (c >= n ? c - n : c);
}

}  // namespace mdlg
