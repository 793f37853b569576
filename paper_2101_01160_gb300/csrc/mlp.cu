// The f_eq surrogate (a project addition, not in the paper): an MLP mapping
// the state point (phi, T, Delta t_LG, Delta x) to the probabilities of the
// (2W+1)^2 = 81 displacement classes, trained on histograms measured by the
// MD of this library.  Hidden layers are BF16 GEMMs on the tensor cores
// (tcgen05.mma, FP32 accumulation in TMEM, fused bias/activation epilogues);
// the 4-input first layer, softmax, loss, transposes, bias gradients and
// Adam are CUDA-core kernels.
//
// Model: x_f = (x - shift)/scale; h_1 = silu(W_1 x_f + b_1) (CUDA cores);
// h_l = silu(W_l h_{l-1} + b_l), l = 2..L-1 (tensor cores); logits =
// W_L h_{L-1} + b_L (tensor cores, classes padded to 128 with zero rows);
// p = softmax(logits[0..81)); loss = mean D_KL(t || p).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "umma.cuh"

namespace mdlg {

using bf16 = __nv_bfloat16;

constexpr int GBM = 128;   // GEMM tile rows (TMEM lanes)
constexpr int GBK = 64;    // K per pipeline stage
constexpr int GRAD_MAX_SPLIT = 64;   // K splits of a weight-gradient GEMM (K = the batch)
constexpr uint64_t GEMM_WAIT_NS = 2000000000ull;

enum Epi { EPI_F32 = 0, EPI_BIAS_F32 = 1, EPI_BIAS_SILU = 2, EPI_DSILU = 3 };

struct GemmArgs {
    const bf16 *A;      // [M][K] row-major (K contiguous)
    const bf16 *B;      // [N][K] row-major
    int lda, ldb, M, N, K;
    float *C;           // FP32 output (EPI_F32 / EPI_BIAS_F32; pre-activation for EPI_BIAS_SILU)
    int ldc;
    long long c_split;  // EPI_F32 split over K (grid.y = z): K range z of length K, tile at C + z c_split
    bf16 *H;            // BF16 output (activation or gradient)
    int ldh;
    const float *bias;  // [N]
    const float *Zp;    // EPI_DSILU: pre-activation, [M][ldz]
    int ldz;
    int *status;
    uint64_t wait_ns;   // limit of every mbarrier wait (0: GEMM_WAIT_NS)
    int dbg_skip_commit;   // bf16_gemm_selftest: CTA 0 does not signal stage dbg_skip_commit - 1 (0: never)
};

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void cpa16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(umma::saddr(dst)), "l"(src) : "memory");
}

// Byte offset of element (row r, k) of a K-major tile of GBK columns in the
// no-swizzle core-matrix layout: 8x8 blocks of 128 bytes, blocks along K
// adjacent (LBO = 128 B), 8-row groups GBK/8 blocks apart (SBO = 1024 B).
__device__ __forceinline__ int tile_off(int r, int k8) { return (r >> 3) * 1024 + k8 * 128 + (r & 7) * 16; }

// C = A * B^T on the tensor cores; one CTA computes a 128 x N tile (N <= 256,
// a multiple of 16) with the accumulator in N TMEM columns.  K is consumed
// in stages of 64: the loads of stage k+1 overlap the MMAs of stage k.
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = g.N;
    const int a_bytes = GBM * GBK * 2, b_bytes = N * GBK * 2;
    unsigned char *st0 = sm, *st1 = sm + a_bytes + b_bytes;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 2 * (a_bytes + b_bytes));
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(mbar + 3);   // mbar[2]: drain after a failed wait
    __shared__ int s_ok;
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
    const uint64_t wait_ns = g.wait_ns ? g.wait_ns : GEMM_WAIT_NS;
    if (warp == 0) umma::tmem_alloc(s_tmem, ncols);
    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        umma::mbar_init(&mbar[2], 1);
        umma::mbar_fence_init();
        s_ok = 1;
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *s_tmem;
    const int m0 = blockIdx.x * GBM;
    const int nk = g.K / GBK;
    const int kb = (int)blockIdx.y * nk;   // first stage of this CTA's K range
    const int n0 = (int)blockIdx.z * N;    // first output column of this CTA (N split)
    const uint32_t idesc = umma::idesc_bf16(GBM, N);
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        unsigned char *sa = s ? st1 : st0;
        unsigned char *sb = sa + a_bytes;
        if (kt >= 2 && !umma::mbar_wait(&mbar[s], ((kt - 2) >> 1) & 1, wait_ns)) s_ok = 0;
        __syncthreads();
        if (!s_ok) break;
        for (int c = tid; c < GBM * 8; c += 128) {
            const int r = c >> 3, k8 = c & 7;
            cpa16(sa + tile_off(r, k8), g.A + (size_t)(m0 + r) * g.lda + (kb + kt) * GBK + k8 * 8);
        }
        for (int c = tid; c < N * 8; c += 128) {
            const int r = c >> 3, k8 = c & 7;
            cpa16(sb + tile_off(r, k8), g.B + (size_t)(n0 + r) * g.ldb + (kb + kt) * GBK + k8 * 8);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        umma::fence_proxy_smem();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after();
            const uint32_t a0 = umma::saddr(sa), b0 = umma::saddr(sb);
#pragma unroll
            for (int k4 = 0; k4 < GBK / 16; ++k4)
                umma::mma(tmem, umma::desc(a0 + k4 * 256, 128, 1024), umma::desc(b0 + k4 * 256, 128, 1024),
                          idesc, (kt | k4) ? 1u : 0u);
            // the self-test withholds one signal so that a later wait runs out
            if (!(g.dbg_skip_commit == kt + 1 && blockIdx.x == 0)) umma::commit(&mbar[s]);
        }
    }
    if (s_ok) {
        const int last = nk - 1;
        if (!umma::mbar_wait(&mbar[last & 1], (last >> 1) & 1, wait_ns)) s_ok = 0;
    }
    if (!s_ok && tid == 0) {
        // a wait gave up: the MMAs this CTA issued may still run; wait (with a
        // limit) until they are done before their TMEM is freed
        umma::commit(&mbar[2]);
        umma::mbar_wait(&mbar[2], 0, wait_ns);
    }
    __syncthreads();
    umma::fence_after();
    if (s_ok) {
        const int row = m0 + warp * 32 + lane;
        for (int cl = 0; cl < N; cl += 16) {
            float v[16];
            umma::ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cl, v);
            const int c0 = n0 + cl;   // output column
            if (EPI == EPI_F32 || EPI == EPI_BIAS_F32) {
                float4 *dst = reinterpret_cast<float4 *>(g.C + (size_t)blockIdx.y * g.c_split + (size_t)row * g.ldc + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float4 o;
                    o.x = v[4 * q + 0] + (EPI == EPI_BIAS_F32 ? g.bias[c0 + 4 * q + 0] : 0.0f);
                    o.y = v[4 * q + 1] + (EPI == EPI_BIAS_F32 ? g.bias[c0 + 4 * q + 1] : 0.0f);
                    o.z = v[4 * q + 2] + (EPI == EPI_BIAS_F32 ? g.bias[c0 + 4 * q + 2] : 0.0f);
                    o.w = v[4 * q + 3] + (EPI == EPI_BIAS_F32 ? g.bias[c0 + 4 * q + 3] : 0.0f);
                    dst[q] = o;
                }
            } else {
                __align__(16) bf16 hb[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float o;
                    if (EPI == EPI_BIAS_SILU) {
                        const float z = v[i] + g.bias[c0 + i];
                        if (g.C) g.C[(size_t)row * g.ldc + c0 + i] = z;
                        o = silu(z);
                    } else {
                        o = v[i] * silu_grad(g.Zp[(size_t)row * g.ldz + c0 + i]);
                    }
                    hb[i] = __float2bfloat16_rn(o);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(g.H + (size_t)row * g.ldh + c0);
                dst[0] = reinterpret_cast<const uint4 *>(hb)[0];
                dst[1] = reinterpret_cast<const uint4 *>(hb)[1];
            }
        }
    } else if (tid == 0) {
        atomicOr(g.status, 1);
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tmem, ncols);
}

size_t gemm_smem(int N) { return 2 * (size_t)(GBM * GBK * 2 + N * GBK * 2) + 32; }

// ksplit > 1 (EPI_F32 only): g.K is one split's K; split z writes its
// partial tile to C + z c_split, to be summed in split order.  A GEMM with
// fewer 128-row tiles than the device has SMs is also split over N into two
// column blocks of N/2 (grid.z), each CTA with its own accumulator; the
// arithmetic of every output is the same.
template <int EPI>
int gemm_launch(const GemmArgs &g, cudaStream_t st, int ksplit = 1) {
    if (g.M % GBM || g.K % GBK || g.N % 16 || g.N < 16 || g.N > 256 || g.lda % 8 || g.ldb % 8)
        return fail(MD_E_ARG, "gemm: M %% 128, K %% 64, N %% 16 in [16,256], lda/ldb %% 8 required");
    if (ksplit < 1 || (ksplit > 1 && EPI != EPI_F32)) return fail(MD_E_ARG, "gemm: K split only for EPI_F32");
    int dev = 0, nsm = 0;
    MD_CUDA_TRY(cudaGetDevice(&dev));
    MD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int nsplit = (g.N % 32 == 0 && (long long)(g.M / GBM) * ksplit < nsm) ? 2 : 1;
    GemmArgs gg = g;
    gg.N = g.N / nsplit;
    const size_t smem = gemm_smem(gg.N);
    MD_CUDA_TRY(cudaFuncSetAttribute(k_gemm<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_gemm<EPI><<<dim3(g.M / GBM, ksplit, nsplit), 128, smem, st>>>(gg);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// ---------------------------------------------------------------- CUDA-core kernels
// First layer (4 inputs): features, pre-activation (optional) and BF16
// activation; rows >= M (padding) get zero features.
__global__ void k_layer1(const float *X, int M, int Mpad, const float *W, const float *b,
                         const float4 shift, const float4 scale, int width, float *xf, float *Z,
                         bf16 *H) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)Mpad * width) return;
    const int m = (int)(i / width), o = (int)(i % width);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
    if (m < M) {
        f0 = (X[4 * m + 0] - shift.x) / scale.x;
        f1 = (X[4 * m + 1] - shift.y) / scale.y;
        f2 = (X[4 * m + 2] - shift.z) / scale.z;
        f3 = (X[4 * m + 3] - shift.w) / scale.w;
    }
    if (xf && o == 0) {
        xf[4 * m + 0] = f0;
        xf[4 * m + 1] = f1;
        xf[4 * m + 2] = f2;
        xf[4 * m + 3] = f3;
    }
    const float z = b[o] + W[4 * o + 0] * f0 + W[4 * o + 1] * f1 + W[4 * o + 2] * f2 + W[4 * o + 3] * f3;
    if (Z) Z[i] = z;
    H[i] = __float2bfloat16_rn(silu(z));
}

// Softmax over the first ncls logits of each row; with targets, also the
// row's share of the mean KL loss and d loss / d logits = (p sum(t) - t) / Mb
// as BF16 (zero in the padding columns).
__global__ void k_softmax(const float *logits, int ldl, int M, int ncls, float *P, const float *T,
                          float *rowloss, bf16 *dlog, int ldd, float inv_batch) {
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (m >= M) return;
    const float *l = logits + (size_t)m * ldl;
    float mx = -INFINITY;
    for (int c = lane; c < ncls; c += 32) mx = fmaxf(mx, l[c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float s = 0.f;
    for (int c = lane; c < ncls; c += 32) s += __expf(l[c] - mx);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const float inv = 1.0f / s;
    float ts = 0.f, loss = 0.f;
    if (T)
        for (int c = lane; c < ncls; c += 32) ts += T[(size_t)m * ncls + c];
    for (int o = 16; o > 0; o >>= 1) ts += __shfl_xor_sync(0xffffffffu, ts, o);
    for (int c = lane; c < ldd || c < ncls; c += 32) {
        if (c < ncls) {
            const float p = __expf(l[c] - mx) * inv;
            if (P) P[(size_t)m * ncls + c] = p;
            if (T) {
                const float t = T[(size_t)m * ncls + c];
                if (t > 0.f) loss += t * (__logf(t) - __logf(p));
                if (dlog) dlog[(size_t)m * ldd + c] = __float2bfloat16_rn((p * ts - t) * inv_batch);
            }
        } else if (dlog && c < ldd) {
            dlog[(size_t)m * ldd + c] = __float2bfloat16_rn(0.f);
        }
    }
    if (rowloss) {
        for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
        if (lane == 0) rowloss[m] = loss * inv_batch;
    }
}

// BF16 transpose [R][C] -> [C][R] through a 32x33 shared tile.
__global__ void k_transpose(const bf16 *in, int R, int C, bf16 *out) {
    __shared__ bf16 t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        t[y][threadIdx.x] = (r < R && c < C) ? in[(size_t)r * C + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (c < C && r < R) out[(size_t)c * R + r] = t[threadIdx.x][y];
    }
}

// Column sums of a BF16 [M][N] matrix in FP32 (fixed order), into out[n].
// Reductions over the batch in two passes with a fixed order: partial sums
// over chunks of GRAD_ROWS rows (grid.y = chunk), then the chunks summed in
// chunk order (k_sum_parts), so that the batch is spread over many CTAs and
// the result does not depend on the launch.
constexpr int GRAD_ROWS = 128;

// part[chunk][n] = sum of column n of a [M][ld] BF16 matrix over the chunk.
__global__ void k_colsum_part(const bf16 *a, int M, int N, int ld, float *part) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int m0 = blockIdx.y * GRAD_ROWS, m1 = min(M, m0 + GRAD_ROWS);
    float s = 0.f;
    for (int m = m0; m < m1; ++m) s += __bfloat162float(a[(size_t)m * ld + n]);
    part[(size_t)blockIdx.y * N + n] = s;
}

// dW_1 = dZ_1^T x_f (4 inputs): part[chunk][o * 4 + k] over the chunk's rows.
__global__ void k_grad_layer1_part(const bf16 *dZ, int M, int width, const float *xf, float *part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= width * 4) return;
    const int o = i / 4, k = i % 4;
    const int m0 = blockIdx.y * GRAD_ROWS, m1 = min(M, m0 + GRAD_ROWS);
    float s = 0.f;
    for (int m = m0; m < m1; ++m) s += __bfloat162float(dZ[(size_t)m * width + o]) * xf[4 * m + k];
    part[(size_t)blockIdx.y * width * 4 + i] = s;
}

// out[r][c] = sum over z = 0 .. nz-1, in z order, of part[z stride + r ldp + c].
__global__ void k_sum_parts(const float *part, int nz, long long stride, int rows, int cols, int ldp,
                            float *out, int ldo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const int r = (int)(i / cols), c = (int)(i % cols);
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += part[z * stride + (long long)r * ldp + c];
    out[(long long)r * ldo + c] = s;
}

// Adam on FP32 master parameters; refreshes the BF16 copy (and its
// transpose) used by the tensor cores.  rows x cols block of a parameter with
// leading dimension ld; master/m/v/g share that layout.
__global__ void k_adam(float *w, float *mom, float *var, const float *g, int rows, int cols, int ld,
                       float lr, float b1, float b2, float c1, float c2, float eps, bf16 *wb,
                       bf16 *wt, int ldt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    const size_t k = (size_t)r * ld + c;
    const float gr = g[k];
    const float m = b1 * mom[k] + (1.f - b1) * gr;
    const float v = b2 * var[k] + (1.f - b2) * gr * gr;
    mom[k] = m;
    var[k] = v;
    const float nw = w[k] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    w[k] = nw;
    if (wb) wb[k] = __float2bfloat16_rn(nw);
    if (wt) wt[(size_t)c * ldt + r] = __float2bfloat16_rn(nw);
}

__global__ void k_to_bf16(const float *w, int n, bf16 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(w[i]);
}

__global__ void k_sum(const float *a, int n, float *out) {
    __shared__ float s[256];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) acc += a[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s[0];
}


// ---------------------------------------------------------------- fused inference
// Whole forward pass in one persistent, warp-specialised kernel over 128-row
// tiles, two tiles in flight per CTA ("slots") so that the CUDA-core
// epilogue of one slot overlaps the tensor-core MMAs of the other.
//   warp 0 lane 0  producer: streams weight chunks, pre-packed in global
//                  memory in the exact shared-memory layout, with one bulk
//                  copy (TMA) each into a ring of F_STAGES buffers;
//   warp 1 lane 0  MMA issuer: per (tile pair, layer, slot) waits for the
//                  slot's activations, issues tcgen05.mma into the slot's
//                  128 x 256 FP32 accumulator in TMEM, commits;
//   warps 2..17    epilogue, 8 warps per slot: stage the inputs, then per
//                  layer TMEM -> bias + SiLU -> BF16 activations written
//                  back over the slot's tile, or after the last layer a
//                  softmax staged in shared memory and stored coalesced.
// Layer 1 (4 inputs) is one K = 16 MMA on split operands: with
// x = x_hi + x_lo, W = W_hi + W_lo and b = b_hi + b_lo (BF16 parts), the A
// row holds (x_hi, x_lo, x_hi, 1, 1, 0, 0) and the B row (W_hi, W_hi, W_lo,
// b_hi, b_lo, 0, 0), so the FP32 accumulator receives
// x_hi W_hi + x_lo W_hi + x_hi W_lo + b, the affine map up to the x_lo W_lo
// term (relative ~2^-16).  The other layers add their bias the same way: a
// first K = 16 MMA of a row of ones (one 8 x 16 block read with a zero
// row-group stride) with (b_hi, b_lo, 0, ...) initialises the accumulator,
// so the epilogue reads finished pre-activations from TMEM.
// A warp may read only the TMEM lanes 32 (warp mod 4) .. +31, so epilogue
// warp w serves rows 32 (w mod 4) + lane and one half of the columns.
// Every wait is bounded; a wait that gives up sets the status flag and the
// roles wind down (uniformly within a slot) instead of hanging.
constexpr int FK = 64;                     // features per weight chunk
constexpr int F_STAGES = 3;
constexpr int F_SBO_A = 256 / 8 * 128;     // 8-row groups of the 256-wide activation tile
constexpr int F_SBO_B = FK / 8 * 128;      // 8-row groups of a weight chunk
constexpr int F_SBO_B0 = 16 / 8 * 128;     // 8-row groups of the K = 16 layer-1 operand
constexpr int F_CHUNK_BYTES = 256 * FK * 2;
constexpr int F_MAXL = 15;
constexpr int F_EPI_WARPS = 8;             // per slot
constexpr int F_THREADS = (2 + 2 * F_EPI_WARPS) * 32;
constexpr int F_ACT_BYTES = 128 * 256 * 2;
constexpr int F_RED_OFF = 60 * 1024;       // softmax partials inside a slot's tile
constexpr int MLP_MAX_CLASSES = 112;       // FP32 stage rows must end below them

struct FusedArgs {
    const float *X;
    long long M;
    float *P;
    int ncls;
    float4 shift, scale;
    const bf16 *Wp[F_MAXL + 1];    // packed operand of every layer (layer 0: split K = 16 with bias)
    const bf16 *Bp[F_MAXL + 1];    // packed bias operand (N x 16) of layers >= 1
    int nt;                        // layers; the last one is the output
    int p_aligned;                 // P 16-byte aligned: output tiles by bulk copy
    int *status;
};

__device__ __forceinline__ int act_off(int r, int k) {
    return (r >> 3) * F_SBO_A + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// silu(z) = z sigmoid(z) = h + h tanh(h), h = z / 2: one special-function
// operation (tanh.approx, relative error about 2^-11, below the BF16 rounding
// of the stored activation) and one FMA.  The hidden layers' packed weights
// and biases are scaled by 1/2 (exact: a power of two), so the accumulator
// already holds h, bit for bit the half of the unscaled pre-activation.
__device__ __forceinline__ float silu_of_half(float h) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// ring chunks of layer l: layer 0 one K = 16 chunk; the others a bias
// chunk (N x 16) followed by the weight chunks
__device__ __forceinline__ int layer_chunks(int l) { return l == 0 ? 1 : 1 + 256 / FK; }

__global__ void __launch_bounds__(F_THREADS, 1) k_mlp_fused(FusedArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *ring = sm + 2 * F_ACT_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + F_STAGES * F_CHUNK_BYTES);
    uint64_t *empty = full + F_STAGES;
    uint64_t *accf = empty + F_STAGES;     // per slot: accumulator complete
    uint64_t *actr = accf + 2;             // per slot: activations written, TMEM read
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(actr + 2);
    unsigned char *ones = reinterpret_cast<unsigned char *>(s_tmem + 4);   // 8 x 16 BF16 block
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 1) umma::tmem_alloc(s_tmem, 512);
    if (tid < 128) {
        // BF16 element e of the block is (r, k) = ((e % 64) / 8, 8 (e / 64) + e % 8)
        const int k = (tid >> 6) * 8 + (tid & 7);
        reinterpret_cast<bf16 *>(ones)[tid] = __float2bfloat16_rn(k < 2 ? 1.f : 0.f);
    }
    umma::fence_proxy_smem();
    if (tid == 0) {
        for (int i = 0; i < F_STAGES; ++i) {
            umma::mbar_init(&full[i], 1);
            umma::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            umma::mbar_init(&accf[i], 1);
            umma::mbar_init(&actr[i], 32 * F_EPI_WARPS);
        }
        umma::mbar_fence_init();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = *s_tmem;
    const long long ntiles = (a.M + 127) / 128;
    const long long my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long npairs = (my_tiles + 1) / 2;
    const int nt = a.nt;
    bool bad = false;

    if (warp == 0) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0;          // phase of the ring pass that stage st is in
            long long c = 0;          // chunks issued
            for (long long p = 0; p < npairs && !bad; ++p)
                for (int l = 0; l < nt && !bad; ++l)
                    for (int s = 0; s < 2 && !bad; ++s) {
                        if (2 * p + s >= my_tiles) continue;
                        const int N = l == nt - 1 ? 128 : 256;
                        for (int kc = 0; kc < layer_chunks(l); ++kc, ++c) {
                            const bool small = l == 0 || kc == 0;     // K = 16 chunk
                            const uint32_t bytes = (uint32_t)(N * (small ? 16 : FK) * 2);
                            const bf16 *srcp = l == 0 ? a.Wp[0] : kc == 0 ? a.Bp[l] : a.Wp[l] + (size_t)(kc - 1) * N * FK;
                            // from the second pass on, wait until the MMAs of
                            // the previous pass have released the stage
                            if (c >= F_STAGES && !umma::mbar_wait(&empty[st], ph ^ 1u, GEMM_WAIT_NS)) {
                                bad = true;
                                break;
                            }
                            umma::mbar_expect_tx(&full[st], bytes);
                            umma::bulk_g2s(ring + st * F_CHUNK_BYTES, srcp, bytes, &full[st]);
                            if (++st == F_STAGES) {
                                st = 0;
                                ph ^= 1u;
                            }
                        }
                    }
            // every copy issued must have landed before the CTA exits: the
            // last min(c, F_STAGES) chunks, walking the ring backwards
            for (long long i = 0; i < c && i < F_STAGES; ++i) {
                if (--st < 0) {
                    st = F_STAGES - 1;
                    ph ^= 1u;
                }
                if (!umma::mbar_wait(&full[st], ph, GEMM_WAIT_NS)) bad = true;
            }
            if (bad) atomicOr(a.status, 1);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0;
            long long c = 0;          // chunks consumed
            int last_st = 0;
            uint32_t last_ph = 0;
            const uint64_t ring_desc = umma::desc(umma::saddr(ring), 128, F_SBO_B);
            const uint64_t ring_desc0 = umma::desc(umma::saddr(ring), 128, F_SBO_B0);
            const uint64_t ones_desc = umma::desc(umma::saddr(ones), 128, 0);   // every row group: the same 8 rows
            uint32_t kpar[2] = {0u, 0u};   // per slot: parity of the next actr phase
            for (long long p = 0; p < npairs && !bad; ++p)
                for (int l = 0; l < nt && !bad; ++l)
                    for (int s = 0; s < 2 && !bad; ++s) {
                        if (2 * p + s >= my_tiles) continue;
                        if (!umma::mbar_wait(&actr[s], kpar[s], GEMM_WAIT_NS)) {
                            bad = true;
                            break;
                        }
                        kpar[s] ^= 1u;
                        umma::fence_after();
                        const uint32_t idesc = umma::idesc_bf16(128, l == nt - 1 ? 128 : 256);
                        const uint64_t act_desc = umma::desc(umma::saddr(sm + s * F_ACT_BYTES), 128, F_SBO_A);
                        const uint32_t d = tmem + (uint32_t)(s * 256);
                        for (int kc = 0; kc < layer_chunks(l); ++kc, ++c) {
                            if (!umma::mbar_wait(&full[st], ph, GEMM_WAIT_NS)) {
                                bad = true;
                                break;
                            }
                            umma::fence_after();
                            const uint64_t soff = (uint64_t)((st * F_CHUNK_BYTES) >> 4);
                            if (l == 0) {
                                umma::mma(d, act_desc, ring_desc0 + soff, idesc, 0u);
                            } else if (kc == 0) {
                                umma::mma(d, ones_desc, ring_desc0 + soff, idesc, 0u);     // accumulator = bias
                            } else {
                                const uint64_t adesc = act_desc + (uint64_t)(((kc - 1) * (FK / 8) * 128) >> 4);
#pragma unroll
                                for (int k4 = 0; k4 < FK / 16; ++k4)
                                    umma::mma(d, adesc + (uint64_t)(k4 * 16), ring_desc + soff + (uint64_t)(k4 * 16),
                                              idesc, 1u);
                            }
                            umma::commit(&empty[st]);
                            last_st = st;
                            last_ph = ph;
                            if (++st == F_STAGES) {
                                st = 0;
                                ph ^= 1u;
                            }
                        }
                        if (!bad) umma::commit(&accf[s]);
                    }
            // the last MMAs must be complete before TMEM is released
            if (c > 0 && !umma::mbar_wait(&empty[last_st], last_ph, GEMM_WAIT_NS)) bad = true;
            if (bad) atomicOr(a.status, 1);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue slots
        const int e = warp - 2, s = e / F_EPI_WARPS, half = (e / 4) & 1, quad = warp & 3;
        const int r = quad * 32 + lane, bar_id = 1 + s, nthr = 32 * F_EPI_WARPS;
        const int ew = e % F_EPI_WARPS, ts = ew * 32 + lane;   // warp / thread index within the slot
        unsigned char *act = sm + s * F_ACT_BYTES;
        float *stage = reinterpret_cast<float *>(act);
        float *red = reinterpret_cast<float *>(act + F_RED_OFF);   // [max, sum][2 halves][128 rows]
        const uint32_t trow = tmem + (uint32_t)(s * 256) + ((uint32_t)(quad * 32) << 16);
        const int ncls = a.ncls;
        const int hs = (ncls + 31) / 32 * 16;                   // softmax columns per half
        const int cbeg = half * hs, cend = min(cbeg + hs, ncls);
        uint32_t kpar = 0u;                                     // parity of the next accf phase
        for (long long p = 0; p < npairs; ++p) {
            const long long j = 2 * p + s;
            if (j >= my_tiles) break;
            const long long m0 = (blockIdx.x + j * gridDim.x) * 128;
            // ---- inputs: split (x_hi, x_lo, x_hi, 0) rows of the K = 16 operand
            if (half == 0) {
                uint4 u0 = make_uint4(0, 0, 0, 0), u1 = u0;
                if (m0 + r < a.M) {
                    const float4 x = __ldg(reinterpret_cast<const float4 *>(a.X) + m0 + r);
                    const float f0 = (x.x - a.shift.x) / a.scale.x, f1 = (x.y - a.shift.y) / a.scale.y;
                    const float f2 = (x.z - a.shift.z) / a.scale.z, f3 = (x.w - a.shift.w) / a.scale.w;
                    const __nv_bfloat162 h01 = __floats2bfloat162_rn(f0, f1), h23 = __floats2bfloat162_rn(f2, f3);
                    const float2 g01 = __bfloat1622float2(h01), g23 = __bfloat1622float2(h23);
                    u0.x = *reinterpret_cast<const uint32_t *>(&h01);
                    u0.y = *reinterpret_cast<const uint32_t *>(&h23);
                    u0.z = pack_bf16(f0 - g01.x, f1 - g01.y);
                    u0.w = pack_bf16(f2 - g23.x, f3 - g23.y);
                    u1.x = u0.x;
                    u1.y = u0.y;
                    u1.z = pack_bf16(1.f, 1.f);     // k = 12, 13: the bias columns
                }
                *reinterpret_cast<uint4 *>(act + act_off(r, 0)) = u0;
                *reinterpret_cast<uint4 *>(act + act_off(r, 8)) = u1;
                umma::fence_proxy_smem();
            }
            umma::mbar_arrive(&actr[s]);
            // ---- layers
            for (int l = 0; l < nt && !bad; ++l) {
                const bool ok = umma::mbar_wait(&accf[s], kpar, GEMM_WAIT_NS);
                kpar ^= 1u;
                if (!umma::bar_and(bar_id, nthr, ok)) {
                    bad = true;
                    break;
                }
                umma::fence_after();
                if (l < nt - 1) {
                    // 8 groups of 16 columns; the TMEM load of group g + 1 is
                    // in flight while group g is computed
                    const int cb = half * 128;
                    uint32_t v[2][16];
                    umma::ld16_async(trow + (uint32_t)cb, v[0]);
                    umma::wait_ld(v[0]);
#pragma unroll
                    for (int g = 0; g < 8; ++g) {
                        const int cur = g & 1, nxt = cur ^ 1;
                        if (g < 7) umma::ld16_async(trow + (uint32_t)(cb + 16 * (g + 1)), v[nxt]);
                        uint32_t hv[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            hv[i] = pack_bf16(silu_of_half(__uint_as_float(v[cur][2 * i])),
                                              silu_of_half(__uint_as_float(v[cur][2 * i + 1])));
                        *reinterpret_cast<uint4 *>(act + act_off(r, cb + 16 * g)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4 *>(act + act_off(r, cb + 16 * g + 8)) = make_uint4(hv[4], hv[5], hv[6], hv[7]);
                        if (g < 7) umma::wait_ld(v[nxt]);
                    }
                    umma::fence_before();
                    umma::fence_proxy_smem();
                    umma::mbar_arrive(&actr[s]);
                } else {
                    // softmax: each half takes columns [cbeg, cend); row
                    // maxima and sums are combined through shared memory; the
                    // normalised rows are staged densely (stride ncls) over
                    // the slot's tile, which is then one contiguous block of
                    // P, written by a single bulk copy (TMA)
                    float mx = -INFINITY;
                    for (int c0 = cbeg; c0 < cend; c0 += 16) {
                        uint32_t v[16];
                        umma::ld16_async(trow + (uint32_t)c0, v);
                        umma::wait_ld(v);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < cend) mx = fmaxf(mx, __uint_as_float(v[i]));
                    }
                    red[half * 128 + r] = mx;
                    umma::bar_sync(bar_id, nthr);
                    mx = fmaxf(red[r], red[128 + r]);
                    float sum = 0.f;
                    for (int c0 = cbeg; c0 < cend; c0 += 16) {
                        uint32_t v[16];
                        umma::ld16_async(trow + (uint32_t)c0, v);
                        umma::wait_ld(v);
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < cend) {
                                const float ez = __expf(__uint_as_float(v[i]) - mx);
                                sum += ez;
                                stage[r * ncls + c0 + i] = ez;
                            }
                    }
                    umma::fence_before();
                    red[256 + half * 128 + r] = sum;
                    umma::bar_sync(bar_id, nthr);
                    const float inv = 1.0f / (red[256 + r] + red[384 + r]);
                    for (int c = cbeg; c < cend; ++c) stage[r * ncls + c] *= inv;
                    umma::fence_proxy_smem();
                    umma::bar_sync(bar_id, nthr);
                    if (ts == 0) {
                        const long long rows = a.M - m0 < 128 ? a.M - m0 : 128;
                        const uint32_t n = (uint32_t)rows * (uint32_t)ncls, n4 = n & ~3u;
                        float *dst = a.P + (size_t)m0 * ncls;
                        if (a.p_aligned) {
                            if (n4) umma::bulk_s2g(dst, stage, n4 * 4);
                            umma::bulk_commit();
                            for (uint32_t i = n4; i < n; ++i) dst[i] = stage[i];
                            umma::bulk_wait_read();
                        } else {
                            for (uint32_t i = 0; i < n; ++i) dst[i] = stage[i];
                        }
                    }
                    umma::bar_sync(bar_id, nthr);    // the next tile's inputs overwrite the stage
                }
            }
            if (bad) break;
        }
        if (ts == 0) {
            umma::bulk_wait();              // the output rows have reached global memory
            if (bad) atomicOr(a.status, 1);
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 1) umma::tmem_free(tmem, 512);
}

constexpr size_t FUSED_SMEM = 2 * F_ACT_BYTES + F_STAGES * F_CHUNK_BYTES + (2 * F_STAGES + 4) * 8 + 16 + 256;
static_assert(FUSED_SMEM <= 232448, "fused MLP shared memory above 227 KB");
static_assert(128 * MLP_MAX_CLASSES * 4 <= F_RED_OFF && F_RED_OFF + 4 * 128 * 4 <= F_ACT_BYTES,
              "softmax stage overlaps the partials");

// Splits v into BF16 parts: part 0 = bf16(v), part 1 = bf16(v - part 0).
__device__ __forceinline__ float split_part(float v, int part) {
    const float hi = __bfloat162float(__float2bfloat16_rn(v));
    return part == 0 ? hi : v - hi;
}

// The packing kernels below multiply a hidden layer's operands by sc = 1/2
// (the output layer's by 1), which is exact for BF16 values: the fused
// kernel's accumulator then holds half the pre-activation (silu_of_half).

// Packs layer 1, W [256][4] and b [256] FP32, into the split K = 16 operand
// (W_hi, W_hi, W_lo, b_hi, b_lo, 0, 0) in the shared-memory layout.
__global__ void k_pack0(const float *W, const float *b, float sc, bf16 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 256 * 16) return;
    const int n = i / 16, k = i % 16;
    float v = 0.f;
    if (k < 12) v = split_part(W[n * 4 + (k & 3)], k < 8 ? 0 : 1);
    else if (k < 14) v = split_part(b[n], k - 12);
    out[(n >> 3) * (F_SBO_B0 / 2) + (k >> 3) * 64 + (n & 7) * 8 + (k & 7)] = __float2bfloat16_rn(sc * v);
}

// Packs the bias b [N] into the K = 16 operand (b_hi, b_lo, 0, ...).
__global__ void k_packb(const float *b, int N, float sc, bf16 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 16) return;
    const int n = i / 16, k = i % 16;
    const float v = k < 2 ? split_part(b[n], k) : 0.f;
    out[(n >> 3) * (F_SBO_B0 / 2) + (k >> 3) * 64 + (n & 7) * 8 + (k & 7)] = __float2bfloat16_rn(sc * v);
}

// Packs W [N][256] (BF16 row-major) into 64-feature chunks laid out exactly
// as the fused kernel's shared-memory weight buffer.
__global__ void k_pack(const bf16 *W, int N, float sc, bf16 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * 256) return;
    const int n = i / 256, k = i % 256, kc = k / FK, kk = k % FK;
    out[(size_t)kc * N * FK + (n >> 3) * (F_SBO_B / 2) + (kk >> 3) * 64 + (n & 7) * 8 + (kk & 7)] =
        __float2bfloat16_rn(sc * __bfloat162float(W[i]));
}

}  // namespace mdlg

using namespace mdlg;

// ---------------------------------------------------------------- model
struct mlp_model {
    int nl = 0;                   // linear layers (hidden + 1)
    int width = 256, ncls = 81, npad = 128, nin = 4;
    float shift[4], scale[4];
    std::vector<int> out, in, outp;   // per layer l = 0..nl-1 (out padded in outp)
    // FP32 master, Adam moments, gradients: per layer W [outp][in], b [outp]
    std::vector<float *> W, b, mW, vW, mb, vb, gW, gb;
    std::vector<bf16 *> Wh, Wt;   // BF16 [outp][in] and [in][outp] (layers >= 1)
    std::vector<bf16 *> Wp;       // chunk-packed copies for the fused forward pass
    std::vector<bf16 *> Bp;       // packed bias operands (layers >= 1)
    bool packed = false;
    int adam_t = 0;
    // workspace
    long long cap = 0;            // rows
    float *xf = nullptr, *logits = nullptr, *rowloss = nullptr;
    std::vector<float *> Z;       // [cap][width] per hidden layer
    std::vector<bf16 *> H;        // [cap][width] per hidden layer
    bf16 *dA = nullptr, *dB = nullptr, *dlog = nullptr, *tA = nullptr, *tB = nullptr;
    float *part = nullptr;        // partial sums of the batch reductions of the gradients
    int *status = nullptr;
    std::vector<void *> allocs, ws;
};

namespace {

int malloc_into(std::vector<void *> &v, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return fail(MD_E_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    v.push_back(*p);
    return MD_OK;
}

// Grows the row workspace to hold `rows` rows (multiple of 128).
int ensure_ws(mlp_model *m, long long rows) {
    if (rows <= m->cap) return MD_OK;
    cudaDeviceSynchronize();
    for (void *p : m->ws) cudaFree(p);
    m->ws.clear();
    const size_t R = (size_t)rows, Wd = (size_t)m->width;
    int rc = MD_OK;
    auto A = [&](void **p, size_t bytes) {
        if (rc == MD_OK) rc = malloc_into(m->ws, p, bytes);
    };
    A((void **)&m->xf, R * 4 * sizeof(float));
    A((void **)&m->logits, R * m->npad * sizeof(float));
    A((void **)&m->rowloss, R * sizeof(float));
    m->Z.assign(m->nl - 1, nullptr);
    m->H.assign(m->nl - 1, nullptr);
    for (int l = 0; l < m->nl - 1; ++l) {
        A((void **)&m->Z[l], R * Wd * sizeof(float));
        A((void **)&m->H[l], R * Wd * sizeof(bf16));
    }
    A((void **)&m->dA, R * Wd * sizeof(bf16));
    A((void **)&m->dB, R * Wd * sizeof(bf16));
    A((void **)&m->dlog, R * m->npad * sizeof(bf16));
    A((void **)&m->tA, R * Wd * sizeof(bf16));
    A((void **)&m->tB, R * Wd * sizeof(bf16));
    A((void **)&m->part, std::max((size_t)GRAD_MAX_SPLIT * Wd * Wd,
                                  ((size_t)rows / GRAD_ROWS + 1) * Wd * 4) * sizeof(float));
    if (rc) return rc;
    m->cap = rows;
    return MD_OK;
}

int refresh_bf16(mlp_model *m, cudaStream_t st) {
    m->packed = false;
    for (int l = 1; l < m->nl; ++l) {
        const int n = m->outp[l] * m->in[l];
        k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(m->W[l], n, m->Wh[l]);
        dim3 tb(32, 8), gr((m->in[l] + 31) / 32, (m->outp[l] + 31) / 32);
        k_transpose<<<gr, tb, 0, st>>>(m->Wh[l], m->outp[l], m->in[l], m->Wt[l]);
    }
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// Forward pass on rows [0, Mpad): H_l (and Z_l when keep_z), logits.
int forward(mlp_model *m, const float *X, long long M, long long Mpad, bool keep_z, cudaStream_t st) {
    const float4 sh = make_float4(m->shift[0], m->shift[1], m->shift[2], m->shift[3]);
    const float4 sc = make_float4(m->scale[0], m->scale[1], m->scale[2], m->scale[3]);
    const long long n1 = Mpad * m->width;
    k_layer1<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(X, (int)M, (int)Mpad, m->W[0], m->b[0], sh,
                                                          sc, m->width, m->xf,
                                                          keep_z ? m->Z[0] : nullptr, m->H[0]);
    MD_CUDA_TRY(cudaGetLastError());
    for (int l = 1; l < m->nl; ++l) {
        GemmArgs g{};
        g.A = m->H[l - 1];
        g.lda = m->width;
        g.B = m->Wh[l];
        g.ldb = m->in[l];
        g.M = (int)Mpad;
        g.N = m->outp[l];
        g.K = m->in[l];
        g.bias = m->b[l];
        g.status = m->status;
        int rc;
        if (l < m->nl - 1) {
            g.C = keep_z ? m->Z[l] : nullptr;
            g.ldc = m->width;
            g.H = m->H[l];
            g.ldh = m->width;
            rc = gemm_launch<EPI_BIAS_SILU>(g, st);
        } else {
            g.C = m->logits;
            g.ldc = m->npad;
            rc = gemm_launch<EPI_BIAS_F32>(g, st);
        }
        if (rc) return rc;
    }
    return MD_OK;
}

// Column sums of dZ [M][N] (bias gradient) over the batch, two passes.
int colsum(const bf16 *dZ, int M, int N, float *part, float *out, cudaStream_t st) {
    const int nch = (M + GRAD_ROWS - 1) / GRAD_ROWS;
    k_colsum_part<<<dim3((N + 127) / 128, nch), 128, 0, st>>>(dZ, M, N, N, part);
    k_sum_parts<<<(N + 255) / 256, 256, 0, st>>>(part, nch, N, 1, N, N, out, N);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

int transpose(const bf16 *in, int R, int C, bf16 *out, cudaStream_t st) {
    dim3 tb(32, 8), gr((C + 31) / 32, (R + 31) / 32);
    k_transpose<<<gr, tb, 0, st>>>(in, R, C, out);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// Loss (device scalar, optional) and gradients of a batch of Mb rows
// (Mb % 128 == 0) into gW / gb.
int backward(mlp_model *m, const float *X, const float *T, int Mb, float *loss_dev, cudaStream_t st) {
    int rc = forward(m, X, Mb, Mb, true, st);
    if (rc) return rc;
    k_softmax<<<(Mb + 7) / 8, 256, 0, st>>>(m->logits, m->npad, Mb, m->ncls, nullptr, T, m->rowloss,
                                            m->dlog, m->npad, 1.0f / (float)Mb);
    MD_CUDA_TRY(cudaGetLastError());
    if (loss_dev) {
        k_sum<<<1, 256, 0, st>>>(m->rowloss, Mb, loss_dev);
        MD_CUDA_TRY(cudaGetLastError());
    }
    // dZ of the current layer (layer L: dlogits) and its width
    const bf16 *dZ = m->dlog;
    int dzw = m->npad;
    bf16 *bufs[2] = {m->dA, m->dB};
    for (int l = m->nl - 1; l >= 1; --l) {
        // dW_l = dZ^T H_{l-1}; db_l = colsum(dZ)
        if ((rc = transpose(dZ, Mb, dzw, m->tA, st))) return rc;
        if ((rc = transpose(m->H[l - 1], Mb, m->width, m->tB, st))) return rc;
        GemmArgs g{};
        g.A = m->tA;
        g.lda = Mb;
        g.B = m->tB;
        g.ldb = Mb;
        g.M = dzw;
        g.N = m->width;
        g.K = Mb;
        g.ldc = m->in[l];
        g.status = m->status;
        // K = the batch: split over up to GRAD_MAX_SPLIT CTAs per tile row
        // (two stages each at least), partial tiles summed in split order
        const int nkt = Mb / GBK;
        int ks = 1;
        while (ks * 2 <= GRAD_MAX_SPLIT && nkt % (ks * 2) == 0 && nkt / (ks * 2) >= 2) ks *= 2;
        if (ks == 1) {
            g.C = m->gW[l];
            if ((rc = gemm_launch<EPI_F32>(g, st))) return rc;
        } else {
            g.K = Mb / ks;
            g.C = m->part;
            g.c_split = (long long)dzw * g.ldc;
            if ((rc = gemm_launch<EPI_F32>(g, st, ks))) return rc;
            const long long n = (long long)dzw * m->width;
            k_sum_parts<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(m->part, ks, g.c_split, dzw, m->width, g.ldc,
                                                                    m->gW[l], g.ldc);
        }
        if ((rc = colsum(dZ, Mb, dzw, m->part, m->gb[l], st))) return rc;
        // dZ_{l-1} = (dZ W_l) * silu'(Z_{l-1})
        GemmArgs d{};
        d.A = dZ;
        d.lda = dzw;
        d.B = m->Wt[l];
        d.ldb = m->outp[l];
        d.M = Mb;
        d.N = m->width;
        d.K = dzw;
        d.H = bufs[l & 1];
        d.ldh = m->width;
        d.Zp = m->Z[l - 1];
        d.ldz = m->width;
        d.status = m->status;
        if ((rc = gemm_launch<EPI_DSILU>(d, st))) return rc;
        dZ = bufs[l & 1];
        dzw = m->width;
    }
    const int nch = (Mb + GRAD_ROWS - 1) / GRAD_ROWS;
    k_grad_layer1_part<<<dim3((m->width * 4 + 127) / 128, nch), 128, 0, st>>>(dZ, Mb, m->width, m->xf, m->part);
    k_sum_parts<<<(m->width * 4 + 255) / 256, 256, 0, st>>>(m->part, nch, (long long)m->width * 4, 1,
                                                            m->width * 4, m->width * 4, m->gW[0], m->width * 4);
    MD_CUDA_TRY(cudaGetLastError());
    return colsum(dZ, Mb, m->width, m->part, m->gb[0], st);
}


}  // namespace

extern "C" {

int mlp_create(int32_t n_hidden, int32_t width, int32_t n_classes, const float *shift4,
               const float *scale4, const float *params, mlp_model **out) {
    if (!out || !shift4 || !scale4 || !params || n_hidden < 2 || n_hidden > 15 || width != 256 ||
        n_classes < 2 || n_classes > MLP_MAX_CLASSES)
        return fail(MD_E_ARG, "mlp_create: n_hidden in [2,15], width 256, classes in [2,112]");
    mlp_model *m = new mlp_model();
    m->nl = n_hidden + 1;
    m->width = width;
    m->ncls = n_classes;
    m->npad = 128;
    std::memcpy(m->shift, shift4, sizeof(m->shift));
    std::memcpy(m->scale, scale4, sizeof(m->scale));
    for (int l = 0; l < m->nl; ++l) {
        m->in.push_back(l == 0 ? 4 : width);
        m->out.push_back(l == m->nl - 1 ? n_classes : width);
        m->outp.push_back(l == m->nl - 1 ? m->npad : width);
    }
    int rc = MD_OK;
    auto A = [&](void **p, size_t bytes) {
        if (rc == MD_OK) rc = malloc_into(m->allocs, p, bytes);
    };
    m->W.assign(m->nl, nullptr);
    m->b = m->mW = m->vW = m->mb = m->vb = m->gW = m->gb = m->W;
    m->Wh.assign(m->nl, nullptr);
    m->Wt.assign(m->nl, nullptr);
    m->Wp.assign(m->nl, nullptr);
    m->Bp.assign(m->nl, nullptr);
    for (int l = 0; l < m->nl; ++l) {
        const size_t nw = (size_t)m->outp[l] * m->in[l], nbias = (size_t)m->outp[l];
        A((void **)&m->W[l], nw * 4);
        A((void **)&m->mW[l], nw * 4);
        A((void **)&m->vW[l], nw * 4);
        A((void **)&m->gW[l], nw * 4);
        A((void **)&m->b[l], nbias * 4);
        A((void **)&m->mb[l], nbias * 4);
        A((void **)&m->vb[l], nbias * 4);
        A((void **)&m->gb[l], nbias * 4);
        if (l > 0) {
            A((void **)&m->Wh[l], nw * 2);
            A((void **)&m->Wt[l], nw * 2);
            A((void **)&m->Wp[l], nw * 2);
            A((void **)&m->Bp[l], (size_t)m->outp[l] * 16 * 2);
        } else {
            A((void **)&m->Wp[0], (size_t)m->outp[0] * 16 * 2);
        }
    }
    A((void **)&m->status, sizeof(int));
    if (rc) {
        mlp_destroy(m);
        return rc;
    }
    for (int l = 0; l < m->nl; ++l) {
        const size_t nw = (size_t)m->outp[l] * m->in[l];
        cudaMemset(m->W[l], 0, nw * 4);
        cudaMemset(m->b[l], 0, m->outp[l] * 4);
        cudaMemset(m->mW[l], 0, nw * 4);
        cudaMemset(m->vW[l], 0, nw * 4);
        cudaMemset(m->mb[l], 0, m->outp[l] * 4);
        cudaMemset(m->vb[l], 0, m->outp[l] * 4);
    }
    cudaMemset(m->status, 0, sizeof(int));
    rc = mlp_set_params(m, params);
    if (rc) {
        mlp_destroy(m);
        return rc;
    }
    *out = m;
    return MD_OK;
}

void mlp_destroy(mlp_model *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    for (void *p : m->ws) cudaFree(p);
    for (void *p : m->allocs) cudaFree(p);
    delete m;
}

int64_t mlp_param_count(mlp_model *m) {
    if (!m) return 0;
    int64_t n = 0;
    for (int l = 0; l < m->nl; ++l) n += (int64_t)m->out[l] * m->in[l] + m->out[l];
    return n;
}

int mlp_set_params(mlp_model *m, const float *params) {
    if (!m || !params) return fail(MD_E_ARG, "mlp_set_params: NULL argument");
    size_t off = 0;
    for (int l = 0; l < m->nl; ++l) {
        const size_t nw = (size_t)m->out[l] * m->in[l];
        MD_CUDA_TRY(cudaMemcpy(m->W[l], params + off, nw * 4, cudaMemcpyDefault));   // rows >= out stay 0
        off += nw;
        MD_CUDA_TRY(cudaMemcpy(m->b[l], params + off, m->out[l] * 4, cudaMemcpyDefault));
        off += m->out[l];
    }
    int rc = refresh_bf16(m, nullptr);
    if (rc) return rc;
    MD_CUDA_TRY(cudaDeviceSynchronize());
    return MD_OK;
}

int mlp_get_params(mlp_model *m, float *params) {
    if (!m || !params) return fail(MD_E_ARG, "mlp_get_params: NULL argument");
    MD_CUDA_TRY(cudaDeviceSynchronize());
    size_t off = 0;
    for (int l = 0; l < m->nl; ++l) {
        const size_t nw = (size_t)m->out[l] * m->in[l];
        MD_CUDA_TRY(cudaMemcpy(params + off, m->W[l], nw * 4, cudaMemcpyDefault));
        off += nw;
        MD_CUDA_TRY(cudaMemcpy(params + off, m->b[l], m->out[l] * 4, cudaMemcpyDefault));
        off += m->out[l];
    }
    return MD_OK;
}

int mlp_forward(mlp_model *m, const float *X, int64_t M, float *P_out, void *stream) {
    mdlg::Range range_("mlp_forward");
    if (!m || !X || !P_out || M < 1) return fail(MD_E_ARG, "mlp_forward: bad arguments");
    if ((uintptr_t)X & 15) return fail(MD_E_ARG, "mlp_forward: X must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (!m->packed) {
        k_pack0<<<16, 256, 0, st>>>(m->W[0], m->b[0], m->nl > 1 ? 0.5f : 1.0f, m->Wp[0]);
        for (int l = 1; l < m->nl; ++l) {
            const int n = m->outp[l] * 256;
            const float sc = l < m->nl - 1 ? 0.5f : 1.0f;
            k_pack<<<(n + 255) / 256, 256, 0, st>>>(m->Wh[l], m->outp[l], sc, m->Wp[l]);
            k_packb<<<(m->outp[l] * 16 + 255) / 256, 256, 0, st>>>(m->b[l], m->outp[l], sc, m->Bp[l]);
        }
        MD_CUDA_TRY(cudaGetLastError());
        m->packed = true;
    }
    FusedArgs a{};
    a.X = X;
    a.M = M;
    a.P = P_out;
    a.ncls = m->ncls;
    a.shift = make_float4(m->shift[0], m->shift[1], m->shift[2], m->shift[3]);
    a.scale = make_float4(m->scale[0], m->scale[1], m->scale[2], m->scale[3]);
    a.nt = m->nl;
    for (int l = 0; l < m->nl; ++l) {
        a.Wp[l] = m->Wp[l];
        a.Bp[l] = m->Bp[l];
    }
    a.p_aligned = ((uintptr_t)P_out & 15) == 0;
    a.status = m->status;
    int dev = 0, nsm = 0;   // the calling thread's current device
    MD_CUDA_TRY(cudaGetDevice(&dev));
    MD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    MD_CUDA_TRY(cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FUSED_SMEM));
    const long long tiles = (M + 127) / 128;
    const int grid = (int)std::min<long long>(tiles, nsm);
    k_mlp_fused<<<grid, F_THREADS, FUSED_SMEM, st>>>(a);
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

int mlp_grad(mlp_model *m, const float *X, const float *T, int32_t B, float *grad_out,
             float *loss_out, void *stream) {
    if (!m || !X || !T || B < 128 || B % 128) return fail(MD_E_ARG, "mlp_grad: batch must be a multiple of 128");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ensure_ws(m, B);
    if (rc) return rc;
    if ((rc = backward(m, X, T, B, loss_out, st))) return rc;
    if (grad_out) {
        size_t off = 0;
        for (int l = 0; l < m->nl; ++l) {
            const size_t nw = (size_t)m->out[l] * m->in[l];
            MD_CUDA_TRY(cudaMemcpyAsync(grad_out + off, m->gW[l], nw * 4, cudaMemcpyDefault, st));
            off += nw;
            MD_CUDA_TRY(cudaMemcpyAsync(grad_out + off, m->gb[l], m->out[l] * 4, cudaMemcpyDefault, st));
            off += m->out[l];
        }
    }
    return MD_OK;
}

int mlp_train_step(mlp_model *m, const float *X, const float *T, int32_t B, float lr,
                   float *loss_out, void *stream) {
    mdlg::Range range_("mlp_train_step");
    int rc = mlp_grad(m, X, T, B, nullptr, loss_out, stream);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    m->adam_t += 1;
    m->packed = false;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)m->adam_t), c2 = 1.f - powf(b2, (float)m->adam_t);
    for (int l = 0; l < m->nl; ++l) {
        const int rows = m->out[l], cols = m->in[l];
        k_adam<<<(rows * cols + 255) / 256, 256, 0, st>>>(m->W[l], m->mW[l], m->vW[l], m->gW[l], rows,
                                                          cols, cols, lr, b1, b2, c1, c2, eps,
                                                          l ? m->Wh[l] : nullptr,
                                                          l ? m->Wt[l] : nullptr, m->outp[l]);
        k_adam<<<(rows + 255) / 256, 256, 0, st>>>(m->b[l], m->mb[l], m->vb[l], m->gb[l], 1, rows, rows,
                                                   lr, b1, b2, c1, c2, eps, nullptr, nullptr, 0);
    }
    MD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

int mlp_status(mlp_model *m) {
    if (!m) return fail(MD_E_ARG, "mlp_status: NULL model");
    int s = 0;
    MD_CUDA_TRY(cudaDeviceSynchronize());
    MD_CUDA_TRY(cudaMemcpy(&s, m->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (s) {
        cudaMemset(m->status, 0, sizeof(int));
        return fail(MD_E_TIMEOUT, "tensor-core GEMM wait timed out");
    }
    return MD_OK;
}

int bf16_gemm_selftest(const void *A, const void *B, float *C, int32_t M, int32_t N, int32_t K,
                       int32_t *status, double limit_s, void *stream) {
    if (!A || !B || !C || !status || !(limit_s > 0.0) || !(limit_s <= 2.0) || K < 3 * GBK)
        return fail(MD_E_ARG, "bf16_gemm_selftest: bad arguments (K >= 192, 0 < limit_s <= 2)");
    GemmArgs g{};
    g.A = (const bf16 *)A;
    g.B = (const bf16 *)B;
    g.lda = K;
    g.ldb = K;
    g.M = M;
    g.N = N;
    g.K = K;
    g.C = C;
    g.ldc = N;
    g.status = status;
    g.wait_ns = (uint64_t)(limit_s * 1e9);
    g.dbg_skip_commit = 1;   // stage 0
    cudaStream_t st = (cudaStream_t)stream;
    MD_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    int rc = gemm_launch<EPI_F32>(g, st);
    if (rc) return rc;
    int32_t h = 0;
    MD_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st));
    MD_CUDA_TRY(cudaStreamSynchronize(st));
    return h ? fail(MD_E_TIMEOUT, "bf16_gemm_selftest: an mbarrier wait ran out (as intended)") : MD_OK;
}

int bf16_gemm_tn(const void *A, const void *B, float *C, int32_t M, int32_t N, int32_t K,
                 int32_t *status, void *stream) {
    if (!A || !B || !C || !status) return fail(MD_E_ARG, "bf16_gemm_tn: NULL argument");
    GemmArgs g{};
    g.A = (const bf16 *)A;
    g.B = (const bf16 *)B;
    g.lda = K;
    g.ldb = K;
    g.M = M;
    g.N = N;
    g.K = K;
    g.C = C;
    g.ldc = N;
    g.status = status;
    return gemm_launch<EPI_F32>(g, (cudaStream_t)stream);
}

}  // extern "C"
