// Device side of the MD system: data layout, the persistent step kernel and
// the cell-list rebuild.  Included by md.cu only.
//
// Layout (all replicas of a batch back to back):
//   * slots: replica r owns slots [pbase_r, pbase_r + cap_r), cap_r = n_r
//     rounded up to SLOT_PAD; slots past n_r are padding, never active.
//   * particles are sorted by MD cell (row-major cy*nc + cx) within each
//     replica, and by particle id inside a cell; cell_start[cbase_r + c] is
//     the first slot of cell c.  Each replica has one extra "padding cell"
//     after its nc^2 cells that owns its padding slots, so a single exclusive
//     scan over all cells yields every replica's cell_start.
//   * per slot: packed cell (cx | cy << 16), offset from the cell corner
//     (Vec2<T>, double-buffered: step s reads one buffer and writes the
//     other), velocity (Vec2<T>), particle id.  The four arrays come in two
//     sets; a rebuild gathers the sorted particles from one set into the
//     other.
//   * work is cut into chunks of ppt*BLOCK consecutive slots of one replica,
//     in a table ordered by decreasing estimated cost; the first rounds of
//     the table are dealt to CTAs round-robin, the rest claimed at run time
//     (for_each_group); the sort phases and the sampling pass deal all of
//     them round-robin.
//   * Verlet neighbour lists (all particles within rv = rc + skin at the last
//     rebuild, in cell-stencil order), ELL layout interleaved by 32-slot
//     groups: entry k of list position q is nbr[(q/32)*K*32 + k*32 + q%32],
//     so a warp reads one entry for all its lanes in one coalesced access.
//     An entry packs the neighbour's slot and its cell offset (dcx+1,
//     dcy+1).  Staged shapes: position = slot.  Global-memory shapes: the
//     positions of a chunk hold its slots in order of decreasing list
//     batches and nn[q] names the slot (chunk_lists_sorted).  The
//     lists' contents do not depend on the launch shape.
//   * the position window of a chunk is the contiguous (periodically
//     wrapped) slot range holding every particle of the cells from one row
//     below the chunk's first cell to one row above its last cell; each step
//     it is staged in shared memory with asynchronous copies, double
//     buffered so that the next chunk's window arrives while the current
//     chunk is computed.
//   * sampling snapshots are indexed by particle id: packed cell + offset.
#pragma once

#include "common.cuh"
#include "lattice.cuh"

namespace mdlg {

constexpr int SLOT_PAD = 256;   // slot padding per replica (multiple of every block size)
constexpr int GRAN = 128;       // slots per replica-lookup granule
constexpr int MAX_CPC = 128;    // most chunks one CTA may own

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };


struct RepDev {
    int32_t nc, cbase, pbase, n, cap, ibase;
    int32_t lx[MD_MAX_DX];
    double h, L, dt, hk, rc2, eps, sig2, vshift, mass;
    double rv2, half_skin;         // Verlet radius^2, rebuild displacement bound
    double dxl[MD_MAX_DX];
    float dxl_invf[MD_MAX_DX];     // RN32(1 / dxl): the FP32 lattice-cell decision
    float hf, dtf, hkf, rc2f, epsf, sig2f, rv2f;
};

struct Control {
    unsigned bar_count, bar_gen;
    int status;
    int set, cur;
    int pad0;
    long long n_rebuilds;
    unsigned vmax[3];     // global engine: per-step max |v| dt / half_skin (float bits), by step mod 3
    unsigned pad1;
    unsigned long long claims;   // global engine: chunk claims of this launch (zeroed before it)
};

// Everything the kernels need, passed by value.
struct SysDev {
    const RepDev *reps;
    const int32_t *gran_rep;    // replica of each GRAN-slot granule
    const int4 *chunks;         // {rep, first slot, end slot, 0}
    Control *ctl;
    int32_t nslots, nrep, total_cells, nchunks, ppt, K, stage;
    int32_t nstatic;            // chunks [0, nstatic) dealt to CTAs, the rest claimed
    int32_t n_lg, n_dx, W, nb, block_windows;
    long long n_equil;
    int32_t lg_every[MD_MAX_LG];
    // state, [set][slot] and pos [set][buf][slot]
    uint32_t *cell[2];
    int32_t *pid[2];
    void *vel[2];
    void *pos[2][2];
    // cell list and rebuild scratch
    int32_t *cellcnt, *cell_start, *newcell, *rank, *perm, *blocksum;
    uint32_t *nbr;              // [nslots/32][K][32]
    // neighbours of each slot.  Staged shapes: nn[slot] = count, lists in
    // slot order.  Global-memory shapes: the slots of every chunk are laid
    // out in order of decreasing list batches (sorted position q), list q
    // and nn[q] = count | (slot - chunk start) << 16 belong to that slot.
    int32_t *nn;
    int32_t *cnt_id;            // [ntot] by particle id: list length at the last rebuild
    // sampling
    uint32_t *snap_cell;        // [n_lg][ntot] by particle id
    void *snap_off;             // [n_lg][ntot] Vec2<T>
    int32_t *hist;              // [nrep][n_lg][n_dx][MD_NBLK][nb]
    unsigned long long *ovf;    // [nrep][n_lg][n_dx]
    double *mom;                // [nslots/32][n_lg][2]
    // per replica: the step's largest |v| dt / (skin/2) (float bits) by step
    // mod 3 (resident engine), and a bound on any displacement since the
    // replica's cells were last made canonical, in half skins (kept between
    // launches; the global engine keeps one bound for all, their maximum)
    unsigned *vmax_rep;         // [nrep][3]
    double *disp_rep;           // [nrep]
    long long ntot;
    uint64_t timeout_ns;
    // force of the last step's force pass by particle id (md_step_forces), or
    // NULL in ordinary steps
    double *dbg_fx, *dbg_fy;
    // md_barrier_selftest: this CTA leaves the kernel instead of arriving at
    // the first step's grid barrier (-1 in every other launch)
    int32_t dbg_leave_cta;
};

// largest staged position window of a chunk (12 KB FP32, 24 KB FP64)
template <typename T> struct WinParts;
template <> struct WinParts<float> { static constexpr int value = 1536; };
template <> struct WinParts<double> { static constexpr int value = 1536; };

// neighbour-list entry: [31:30] dcy+1, [29:28] dcx+1, [27:0] slot
constexpr uint32_t NB_INDEX = (1u << 28) - 1u;
// list entries per particle read in one batch (and staged in shared memory
// with the chunk): 4 in FP32, 8 in FP64 (fewer register spills at each
// precision's register budget; measured)
template <typename T> constexpr int NB_STAGE = sizeof(T) == 4 ? 4 : 8;

template <typename T> __device__ __forceinline__ T rd(double d, float f);
template <> __device__ __forceinline__ double rd<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float rd<float>(double, float f) { return f; }

// 1/r^2 of a pair: the hardware reciprocal in FP32 (relative error ~1e-7,
// far below the force tolerance), IEEE division in FP64.
__device__ __forceinline__ float inv_r2(float r2) { return __fdividef(1.0f, r2); }
__device__ __forceinline__ double inv_r2(double r2) { return 1.0 / r2; }

// Lennard-Jones sum (Sec. 4: V = 4 eps [(s/r)^12 - (s/r)^6] for r < rc, the
// force being the derivative of the unshifted potential) over slots [a, e)
// of one stencil row whose three cells start at a, m1, m2: the column
// offset of slot j follows from which cell it falls in.  One loop per row
// instead of one per cell keeps the lanes of a warp busier, since their
// candidate counts vary less over a row than over single cells.  pos and
// self refer to the same index space.  Every force evaluation of the
// library goes through this one routine, so the step kernel and the
// observation kernel produce identical bits.
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
// a + b c with the product and the sum rounded separately, never contracted
__device__ __forceinline__ float axpyT(float a, float b, float c) { return __fadd_rn(a, __fmul_rn(b, c)); }
__device__ __forceinline__ double axpyT(double a, double b, double c) { return __dadd_rn(a, __dmul_rn(b, c)); }

// One pair: separation (rx, ry) = x_j - x_i; accumulates the force on i.
// Written with explicit fused multiply-adds so that every caller evaluates
// it with the same roundings.
template <typename T, bool kPE>
__device__ __forceinline__ void lj_pair_acc(T rx, T ry, T rc2, T eps24, T sig2, T &fx, T &fy,
                                            double vshift, double &pe, double &fabs_sum) {
    const T r2 = fmaT(rx, rx, ry * ry);
    if (r2 < rc2) {
        const T ir2 = inv_r2(r2);
        const T s2 = sig2 * ir2;
        const T s6 = s2 * s2 * s2;
        const T fr = eps24 * s6 * fmaT(T(2), s6, T(-1)) * ir2;
        fx = fmaT(-fr, rx, fx);
        fy = fmaT(-fr, ry, fy);
        if (kPE) {
            const double d6 = (double)s6;
            pe += 0.5 * ((double)eps24 / 6.0 * (d6 * d6 - d6) - vshift);
            fabs_sum += fabs((double)fr) * sqrt((double)r2);
        }
    }
}

template <typename T, bool kPE>
__device__ __forceinline__ void lj_row(const typename V2<T>::type *pos, int a, int m1, int m2,
                                       int e, int self, T sxm, T sx0, T sxp, T sy, T rc2,
                                       T eps24, T sig2, T &fx, T &fy, double vshift, double &pe,
                                       double &fabs_sum) {
    for (int j = a; j < e; ++j) {
        if (j == self) continue;
        const typename V2<T>::type o = pos[j];
        const T sx = j < m1 ? sxm : (j < m2 ? sx0 : sxp);
        lj_pair_acc<T, kPE>(o.x + sx, o.y + sy, rc2, eps24, sig2, fx, fy, vshift, pe, fabs_sum);
    }
}

// Force on the particle in slot `self` (packed cell cpk, offset oi) from all
// particles of the 3x3 block of cells around its cell, read from global
// memory.  The separation is (dcx*h + off_j - off_i) per axis: the stencil
// offset dcx carries the periodic image.  Same row/cell order and the same
// arithmetic as lj_window.
template <typename T, bool kPE>
__device__ __forceinline__ void lj_stencil(const RepDev &R, const typename V2<T>::type *pos,
                                           const int32_t *cs, uint32_t cpk,
                                           typename V2<T>::type oi, int self, T &fx, T &fy,
                                           double &pe, double &fabs_sum) {
    const int nc = R.nc;
    const int cx = (int)(cpk & 0xffffu), cy = (int)(cpk >> 16);
    const T h = rd<T>(R.h, R.hf);
    const T rc2 = rd<T>(R.rc2, R.rc2f);
    const T eps24 = T(24) * rd<T>(R.eps, R.epsf);
    const T sig2 = rd<T>(R.sig2, R.sig2f);
    const T sxm = -h - oi.x, sx0 = -oi.x, sxp = h - oi.x;
    const int32_t *csr = cs + R.cbase;
    const bool interior = cx >= 1 && cx <= nc - 2;
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
        const int row = wrap1(cy + oy, nc) * nc;
        const T sy = (T)oy * h - oi.y;
        if (interior) {
            const int c0 = row + cx - 1;
            lj_row<T, kPE>(pos, csr[c0], csr[c0 + 1], csr[c0 + 2], csr[c0 + 3], self, sxm, sx0, sxp,
                           sy, rc2, eps24, sig2, fx, fy, R.vshift, pe, fabs_sum);
        } else {
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int c = row + wrap1(cx + ox, nc);
                const T sx = ox < 0 ? sxm : (ox == 0 ? sx0 : sxp);
                const int e = csr[c + 1];
                lj_row<T, kPE>(pos, csr[c], e, e, e, self, sx, sx, sx, sy, rc2, eps24, sig2, fx, fy,
                               R.vshift, pe, fabs_sum);
            }
        }
    }
}

// ---------------------------------------------------------------- chunk windows
// Window of one chunk, fixed between two rebuilds: U0 = first slot in
// "unwrapped" numbering (slot + k*n across the periodic seam), npw = window
// particles, ok = the window fits the staging buffer.
struct ChunkDesc {
    int start, end, rep, U0, npw, ok, pad0, pad1;
};

__device__ __forceinline__ int unwrapped_start(const int32_t *csr, int c, int nc2, int n) {
    if (c < 0) return csr[c + nc2] - n;
    if (c >= nc2) return csr[c - nc2] + n;
    return csr[c];
}

// Descriptor of chunk ch from the current cell list: cells [cf - nc - 1,
// cl + nc + 1] (circularly), or the whole replica when that is shorter.
__device__ __forceinline__ ChunkDesc make_desc(const SysDev &S, const uint32_t *cell, int ch,
                                               int max_parts) {
    const int4 cd = S.chunks[ch];
    const RepDev &R = S.reps[cd.x];
    const int nc2 = R.nc * R.nc;
    const int32_t *csr = S.cell_start + R.cbase;
    const uint32_t a = cell[cd.y], b = cell[cd.z - 1];
    const int cf = (int)(a >> 16) * R.nc + (int)(a & 0xffffu);
    const int cl = (int)(b >> 16) * R.nc + (int)(b & 0xffffu);
    const int wlen = cl - cf + 2 * R.nc + 3;
    int w0, ncw;
    if (wlen >= nc2) {
        w0 = 0;
        ncw = nc2;
    } else {
        w0 = cf - R.nc - 1;
        ncw = wlen;
    }
    ChunkDesc d;
    d.start = cd.y;
    d.end = cd.z;
    d.rep = cd.x;
    d.U0 = unwrapped_start(csr, w0, nc2, R.n);
    d.npw = unwrapped_start(csr, w0 + ncw, nc2, R.n) - d.U0;
    d.ok = d.npw <= max_parts;
    d.pad0 = d.pad1 = 0;
    return d;
}

// Position of slot j in the window of d, or -1 if outside it.
__device__ __forceinline__ int window_index(const ChunkDesc &d, const RepDev &R, int j) {
    int u = j - d.U0;
    u = u < 0 ? u + R.n : (u >= R.n ? u - R.n : u);
    return u < d.npw ? u : -1;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
template <typename V> __device__ __forceinline__ void cp_async_v(V *dst, const V *src);
template <> __device__ __forceinline__ void cp_async_v<float2>(float2 *d, const float2 *s) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(d)), "l"(s) : "memory");
}
template <> __device__ __forceinline__ void cp_async_v<double2>(double2 *d, const double2 *s) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d)), "l"(s) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void cp_async16(void *d, const void *s) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(d)), "l"(s) : "memory");
}

// Shared-memory staging buffer of one chunk.
template <typename T> struct Stage {
    typename V2<T>::type *pos;   // window positions [WinParts]
    typename V2<T>::type *vel;   // own velocities [chunk]
    int32_t *nn;                 // own neighbour counts [chunk]
    uint32_t *ent;               // own first NB_STAGE entries, [chunk/32][NB_STAGE][32]
};

// Issues the asynchronous copies of chunk d into one staging buffer: window
// positions, own velocities, neighbour counts and the first NB_STAGE list
// entries of every particle.
template <typename T, int BLOCK>
__device__ __forceinline__ void stage_chunk(const SysDev &S, const RepDev &R, const ChunkDesc &d,
                                            const typename V2<T>::type *pin,
                                            const typename V2<T>::type *vel, const Stage<T> &B) {
    const int tid = threadIdx.x;
    if (d.ok) {
        for (int k = tid; k < d.npw; k += BLOCK) {
            int u = d.U0 + k - R.pbase;
            u = u < 0 ? u + R.n : (u >= R.n ? u - R.n : u);
            cp_async_v(&B.pos[k], &pin[R.pbase + u]);
        }
    }
    const int len = d.end - d.start;
    for (int i = tid; i < len; i += BLOCK) cp_async_v(&B.vel[i], &vel[d.start + i]);
    for (int i = 4 * tid; i < len; i += 4 * BLOCK) cp_async16(&B.nn[i], &S.nn[d.start + i]);
    const int ngrp = (len + 31) >> 5;
    const int per = NB_STAGE<T> * 32 / 4;            // 16-byte pieces per group
    for (int t = tid; t < ngrp * per; t += BLOCK) {
        const int g = t / per, r = t % per;
        const uint32_t *src = S.nbr + (long long)((d.start >> 5) + g) * S.K * 32 + r * 4;
        cp_async16(&B.ent[g * NB_STAGE<T> * 32 + r * 4], src);
    }
}

// Chunks are dealt to CTAs round-robin (CTA b owns chunks b, b + G, b + 2G,
// ..., G = gridDim.x) so that dense and sparse replicas mix in every CTA.
__device__ __forceinline__ int own_chunks(int nchunks) {
    return nchunks > (int)blockIdx.x ? (nchunks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
}
__device__ __forceinline__ int own_chunk(int i) { return (int)blockIdx.x + i * (int)gridDim.x; }

// Work distribution of the global-memory shapes: runs body(cd, g0) for every
// 32-slot group of every chunk of one pass, each on exactly one warp (cd the
// chunk, g0 its group's first slot; lanes past the chunk's end have
// slot >= cd.z).  Chunks [0, nstatic) are dealt to CTAs (own_chunk), their
// groups to the CTA's warps in turn.  The rest, the cheapest, are claimed:
// a CTA claims whole chunks from the launch's counter (zeroed before the
// launch) in table order and holds one claimed chunk in reserve; its warps
// take the groups of its current chunk from a shared-memory counter, with no
// CTA-wide sync, so that all CTAs finish the pass within about one group of
// each other.  The warp that takes the group just past the end installs the
// reserve (the first such warp of the pass claims it first) and claims the
// next; warps that overshot wait for the install (shared memory, bounded:
// DS_TIMEOUT after about 2^22 polls).  Every CTA stops claiming at its first
// claim past the table, so a pass issues exactly (nchunks - nstatic) +
// gridDim.x claims and every CTA advances base to the next pass's first value
// without reading the counter; grid barriers separate passes.  Which warp
// computes a group changes no result.
constexpr int GRP_BITS = 10;   // group field of the shared work word
template <int BLOCK, typename F>
__device__ __forceinline__ void for_each_group(const SysDev &S, unsigned long long &base, F &&body) {
    // s_work = (current chunk - nstatic + 1) << GRP_BITS | next group; 0 in
    // the chunk field before the first install, ndyn + 1 once none is left
    __shared__ unsigned s_work;
    __shared__ int s_pend;   // reserve chunk; -1 while its claim is in flight, -2 none yet
    const int nch = S.nchunks, nst = S.nstatic, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ndyn = nch - nst;
    const auto claim = [&]() {
        const unsigned long long v = atomicAdd(&S.ctl->claims, 1ull) - base;
        return v < (unsigned long long)ndyn ? nst + (int)v : nch;
    };
    __syncthreads();   // the previous pass's readers of s_work / s_pend are done
    if (threadIdx.x == 0) {
        s_work = 0u;
        s_pend = -2;
    }
    __syncthreads();
    const int ndealt = own_chunks(nst);
    for (int i = 0; i < ndealt; ++i) {
        const int4 cd = S.chunks[own_chunk(i)];
        const int ng = (cd.z - cd.y + 31) >> 5;
        for (int g = warp; g < ng; g += BLOCK / 32) body(cd, cd.y + 32 * g);
    }
    if (ndyn <= 0) return;
    for (;;) {
        unsigned w = 0;
        if (lane == 0) w = atomicAdd(&s_work, 1u);
        w = __shfl_sync(0xffffffffu, w, 0);
        const int cf = (int)(w >> GRP_BITS), g = (int)(w & ((1u << GRP_BITS) - 1));
        const int c = nst + cf - 1;   // nst - 1: none installed yet
        if (c >= nch) break;
        int4 cd = make_int4(0, 0, 0, 0);
        if (cf > 0) cd = S.chunks[c];
        const int ng = (cd.z - cd.y + 31) >> 5;   // 0 before the first install
        if (g < ng) {
            body(cd, cd.y + 32 * g);
            continue;
        }
        int ok = 1;
        if (lane == 0) {
            unsigned polls = 0;
            if (g == ng) {
                // install the reserve once its claim has landed, then claim anew
                int nc;
                while ((nc = *(volatile int *)&s_pend) == -1 && ++polls < (1u << 22)) __nanosleep(32);
                if (nc == -2) nc = claim();
                if (nc >= 0) {
                    *(volatile int *)&s_pend = -1;
                    __threadfence_block();
                    atomicExch(&s_work, (unsigned)(nc - nst + 1) << GRP_BITS);
                    const int nxt = nc < nch ? claim() : nch;
                    *(volatile int *)&s_pend = nxt;
                } else {
                    ok = 0;
                }
            } else {
                // another warp installs the next chunk
                while ((int)(*(volatile unsigned *)&s_work >> GRP_BITS) == cf && ++polls < (1u << 22))
                    __nanosleep(32);
                ok = polls < (1u << 22);
            }
            if (!ok) atomicOr(&S.ctl->status, (int)DS_TIMEOUT);
        }
        if (!__shfl_sync(0xffffffffu, ok, 0)) break;
    }
    base += (unsigned long long)ndyn + gridDim.x;
}


// ---------------------------------------------------------------- neighbour lists
// Builds the list of slot i from the 3x3 cell stencil (same row/cell order
// as lj_stencil): every j with |x_j - x_i| < rv.  Returns the count; entries
// beyond K are not written and the count reports the overflow.
template <typename T>
__device__ __forceinline__ int build_list(const SysDev &S, const RepDev &R,
                                          const typename V2<T>::type *pos, uint32_t cpk,
                                          typename V2<T>::type oi, int self, int at) {
    const int nc = R.nc;
    const int cx = (int)(cpk & 0xffffu), cy = (int)(cpk >> 16);
    const T h = rd<T>(R.h, R.hf);
    const T rv2 = rd<T>(R.rv2, R.rv2f);
    const int32_t *csr = S.cell_start + R.cbase;
    uint32_t *out = S.nbr + (long long)(at >> 5) * S.K * 32 + (at & 31);   // list position
    int cnt = 0;
    for (int oy = -1; oy <= 1; ++oy) {
        const int row = wrap1(cy + oy, nc) * nc;
        const T sy = (T)oy * h - oi.y;
        for (int ox = -1; ox <= 1; ++ox) {
            const int c = row + wrap1(cx + ox, nc);
            const T sx = (T)ox * h - oi.x;
            const uint32_t tag = ((uint32_t)(ox + 1) << 28) | ((uint32_t)(oy + 1) << 30);
            for (int j = csr[c]; j < csr[c + 1]; ++j) {
                if (j == self) continue;
                const typename V2<T>::type o = pos[j];
                const T rx = o.x + sx, ry = o.y + sy;
                if (rx * rx + ry * ry < rv2) {
                    if (cnt < S.K) out[cnt * 32] = (uint32_t)j | tag;
                    ++cnt;
                }
            }
        }
    }
    return cnt;
}

// Force on slot i from its neighbour list: the same pairs, order and
// arithmetic as lj_stencil (pairs beyond rc contribute nothing), so both
// paths give identical bits.  Neighbours inside the chunk's staged window
// are read from shared memory, the others (column-wrapped neighbours of
// edge particles, chunks without a window) from global memory.
template <typename T>
__device__ __forceinline__ void lj_list_from(const SysDev &S, const RepDev &R, const ChunkDesc &d,
                                             const typename V2<T>::type *spos,
                                             const typename V2<T>::type *pin, typename V2<T>::type oi,
                                             int self, int cnt, uint32_t (&e)[NB_STAGE<T>], T &fx, T &fy) {
    const T h = rd<T>(R.h, R.hf);
    const T rc2 = rd<T>(R.rc2, R.rc2f);
    const T eps24 = T(24) * rd<T>(R.eps, R.epsf);
    const T sig2 = rd<T>(R.sig2, R.sig2f);
    // the shift of a neighbour in column (row) tag t is (t - 1) h - offset:
    // one FMA of the exact factor t - 1 (from the float bits of 2^23 + t,
    // no conversion instruction), the product exact, so the value is the
    // correctly rounded sum the other force paths select from -h - off,
    // -off and h - off (a zero may differ in sign, which moves nothing);
    // two registers instead of six
    const T nox = -oi.x, noy = -oi.y;
    const uint32_t *lst = S.nbr + (long long)(self >> 5) * S.K * 32 + (self & 31);
    double pe_unused = 0.0, fa_unused = 0.0;
    constexpr int U = NB_STAGE<T>;
    // e holds the first batch; each later batch is requested while the
    // previous one is computed.
    for (int k0 = 0; k0 < cnt; k0 += U) {
        uint32_t en[U];
        const bool more = k0 + U < cnt;
        if (more) {
#pragma unroll
            for (int u = 0; u < U; ++u) en[u] = k0 + U + u < cnt ? lst[(k0 + U + u) * 32] : 0u;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (k0 + u < cnt) {
                const int j = (int)(e[u] & NB_INDEX);
                int w = j - d.U0;
                w = w < 0 ? w + R.n : (w >= R.n ? w - R.n : w);
                const typename V2<T>::type o = (d.ok && w < d.npw) ? spos[w] : pin[j];
                const uint32_t ox = (e[u] >> 28) & 3u, oy = e[u] >> 30;
                const float kx = __int_as_float(0x4b000000u | ox) - 8388609.0f;   // ox - 1
                const float ky = __int_as_float(0x4b000000u | oy) - 8388609.0f;
                const T sx = fmaT((T)kx, h, nox);
                const T sy = fmaT((T)ky, h, noy);
                lj_pair_acc<T, false>(o.x + sx, o.y + sy, rc2, eps24, sig2, fx, fy, 0.0, pe_unused,
                                      fa_unused);
            }
        }
        if (more) {
#pragma unroll
            for (int u = 0; u < U; ++u) e[u] = en[u];
        }
    }
}

// lj_list_from with the first batch of list entries read here: without
// waiting for the count (a list holds K >= NB_STAGE entries, so the reads
// stay in bounds; unused ones are masked), from shared memory if staged.
template <typename T>
__device__ __forceinline__ void lj_list(const SysDev &S, const RepDev &R, const ChunkDesc &d,
                                        const typename V2<T>::type *spos, const uint32_t *sent,
                                        const typename V2<T>::type *pin, typename V2<T>::type oi,
                                        int self, int cnt, T &fx, T &fy) {
    uint32_t e[NB_STAGE<T>];
    const uint32_t *lst = S.nbr + (long long)(self >> 5) * S.K * 32 + (self & 31);
#pragma unroll
    for (int u = 0; u < NB_STAGE<T>; ++u) e[u] = sent ? sent[u * 32] : lst[u * 32];
    lj_list_from<T>(S, R, d, spos, pin, oi, self, cnt, e, fx, fy);
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) / 16 * 16; }

// Runs body(chunk) for every chunk of the table on one CTA each (body may
// sync the CTA): CTAs claim chunks from the launch's counter in table order,
// one claim ahead.  Every CTA stops at its first claim past the table, so a
// pass issues exactly nchunks + gridDim.x claims and base advances without a
// read of the counter (the same accounting as for_each_group).
template <typename F>
__device__ __forceinline__ void for_each_chunk_cta(const SysDev &S, unsigned long long &base, F &&body) {
    __shared__ int s_c;
    const int nch = S.nchunks;
    unsigned long long next = 0;
    __syncthreads();   // s_c of an earlier pass is read
    if (threadIdx.x == 0) next = atomicAdd(&S.ctl->claims, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long v = next - base;
            s_c = v < (unsigned long long)nch ? (int)v : nch;
            if (s_c < nch) next = atomicAdd(&S.ctl->claims, 1ull);
        }
        __syncthreads();
        const int c = s_c;
        __syncthreads();   // s_c is rewritten by the next claim
        if (c >= nch) break;
        body(c);
    }
    base += (unsigned long long)nch + gridDim.x;
}

// Shared scratch of the sorted list layout: [chunk / 32 + 1][16] counts and
// chunk 16-bit ranks.
__host__ __device__ inline size_t sort_scratch_bytes(int chunk) {
    return align16((size_t)(chunk / 32 + 1) * 16 * sizeof(int)) + align16((size_t)chunk * sizeof(uint16_t));
}

// Neighbour lists of one chunk in the sorted layout of the global-memory
// shapes (the whole CTA).  A warp's pair loop runs as many list batches as
// its longest list, so the chunk's slots are laid out in order of decreasing
// batches -- estimated by each particle's list length at the previous
// rebuild (cnt_id), the lists moving little between rebuilds -- with ties in
// slot order: a counting sort over 16 batch classes, per 32-slot block a
// warp match for the ranks, one exclusive scan in class-major order.  So
// the layout is deterministic, and each particle's list (its pairs and
// their order) is the same as in slot order: no force changes.
template <typename T, int BLOCK>
__device__ __forceinline__ void chunk_lists_sorted(const SysDev &S, int set, const int4 cd,
                                                   unsigned char *scratch, int &over) {
    using V = typename V2<T>::type;
    const int tid = threadIdx.x, lane = tid & 31, n = cd.z - cd.y;
    const int nwc = (n + 31) >> 5;
    int *hist = reinterpret_cast<int *>(scratch);   // [nwc][16]: counts, then starts
    uint16_t *rk = reinterpret_cast<uint16_t *>(scratch + align16((size_t)(n / 32 + 1) * 16 * sizeof(int)));
    const V *npos = static_cast<const V *>(S.pos[set][0]);
    const uint32_t *ncell = S.cell[set];
    const int32_t *pid = S.pid[set];
    const RepDev &R = S.reps[cd.x];
    for (int i = tid; i < nwc * 16; i += BLOCK) hist[i] = 0;
    __syncthreads();
    for (int b0 = 0; b0 < n; b0 += BLOCK) {   // the same trip count on every thread
        const int i = b0 + tid;
        int cls = 16;                          // no slot
        if (i < n) {
            const int k = S.cnt_id[pid[cd.y + i]];
            cls = 15 - min((k + NB_STAGE<T> - 1) / NB_STAGE<T>, 15);
        }
        const unsigned m = __match_any_sync(0xffffffffu, cls);
        const int r = __popc(m & ((1u << lane) - 1u));
        if (i < n) {
            rk[i] = (uint16_t)(cls << 8 | r);
            if (r == 0) hist[(i >> 5) * 16 + cls] = __popc(m);
        }
    }
    __syncthreads();
    if (tid < 32) {
        // exclusive scan over (class, block) in class-major order, in place
        int carry = 0;
        for (int e0 = 0; e0 < 16 * nwc; e0 += 32) {
            const int e = e0 + lane;
            const int at = e < 16 * nwc ? (e % nwc) * 16 + e / nwc : 0;
            const int v = e < 16 * nwc ? hist[at] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (e < 16 * nwc) hist[at] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    for (int i = tid; i < n; i += BLOCK) {
        const int cls = rk[i] >> 8, r = rk[i] & 255;
        const int q = cd.y + hist[(i >> 5) * 16 + cls] + r;
        const int slot = cd.y + i;
        const int cnt = build_list<T>(S, R, npos, ncell[slot], npos[slot], slot, q);
        const int kept = cnt < S.K ? cnt : S.K;
        S.nn[q] = kept | (i << 16);
        S.cnt_id[pid[slot]] = kept;
        over |= cnt > S.K;
    }
    __syncthreads();   // the scratch is reused by the next chunk
}

// ---------------------------------------------------------------- rebuild
// With mode RB_ALL every particle gets its canonical cell (the MD cell its
// offset now lies in, the offset re-expressed from that cell's corner); with
// RB_NONE every particle keeps its cell (a sort of a state written in
// another order).  Then a counting sort of all particles by cell, particles
// inside one cell ordered by id, so the order -- and therefore every force
// sum -- is reproducible and independent of the launch shape; then the
// neighbour lists.  Six grid barriers (seven in the global-memory shapes,
// whose lists other CTAs read next).  Padding slots keep perm = -1 (set at
// creation).
enum RebuildMode { RB_ALL = 1, RB_NONE = 2 };

template <typename T, int BLOCK>
__device__ bool rebuild(const SysDev &S, int &set, int &cur, unsigned &gen, int nloc,
                        ChunkDesc *s_desc, int mode, unsigned long long &claim0,
                        unsigned char *sort_mem) {
    using V = typename V2<T>::type;
    Control *C = S.ctl;
    const GridBarrier bar{&C->bar_count, &C->bar_gen, &C->status};
    const int tid = threadIdx.x;
    const V *pos = static_cast<const V *>(S.pos[set][cur]);
    const uint32_t *cell = S.cell[set];
    // R1: new cell and rank inside it
    for (int i = 0; i < nloc; ++i) {
        const int4 cd = S.chunks[own_chunk(i)];
        const RepDev &R = S.reps[cd.x];
        const T h = rd<T>(R.h, R.hf);
        const bool canon = mode == RB_ALL;
        for (int slot = cd.y + tid; slot < cd.z; slot += BLOCK) {
            const V o = pos[slot];
            const uint32_t cpk = cell[slot];
            const int sx = !canon ? 0 : (o.x >= h ? 1 : (o.x < T(0) ? -1 : 0));
            const int sy = !canon ? 0 : (o.y >= h ? 1 : (o.y < T(0) ? -1 : 0));
            const int ncx = wrap1((int)(cpk & 0xffffu) + sx, R.nc);
            const int ncy = wrap1((int)(cpk >> 16) + sy, R.nc);
            const int gc = R.cbase + ncy * R.nc + ncx;
            S.newcell[slot] = gc;
            S.rank[slot] = atomicAdd(&S.cellcnt[gc], 1);
        }
    }
    if (!grid_sync(bar, gen, S.timeout_ns)) return false;
    // R2: per-CTA sums over a contiguous segment of cells
    const int seg = (S.total_cells + gridDim.x - 1) / gridDim.x;
    const int s0 = min(S.total_cells, (int)blockIdx.x * seg), s1 = min(S.total_cells, s0 + seg);
    __shared__ int s_w[BLOCK / 32];
    __shared__ int s_base;
    {
        int acc = 0;
        for (int c = s0 + tid; c < s1; c += BLOCK) acc += S.cellcnt[c];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) s_w[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < BLOCK / 32; ++w) t += s_w[w];
            S.blocksum[blockIdx.x] = t;
        }
    }
    if (!grid_sync(bar, gen, S.timeout_ns)) return false;
    // R3: exclusive scan into cell_start
    {
        int acc = 0;
        for (int b = tid; b < (int)blockIdx.x; b += BLOCK) acc += S.blocksum[b];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncthreads();
        if ((tid & 31) == 0) s_w[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < BLOCK / 32; ++w) t += s_w[w];
            s_base = t;
        }
        __syncthreads();
        int base = s_base;
        const int lane = tid & 31, wid = tid >> 5;
        for (int c0 = s0; c0 < s1; c0 += BLOCK) {
            const int c = c0 + tid;
            const int v = c < s1 ? S.cellcnt[c] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            __syncthreads();
            if (lane == 31) s_w[wid] = incl;
            __syncthreads();
            int wbase = 0, tile = 0;
            for (int w = 0; w < BLOCK / 32; ++w) {
                if (w < wid) wbase += s_w[w];
                tile += s_w[w];
            }
            if (c < s1) S.cell_start[c] = base + wbase + incl - v;
            base += tile;
        }
        if ((int)blockIdx.x == (int)gridDim.x - 1 && tid == 0) S.cell_start[S.total_cells] = base;
    }
    if (!grid_sync(bar, gen, S.timeout_ns)) return false;
    // R4: scatter slot numbers to their new place; reset counts
    for (int i = 0; i < nloc; ++i) {
        const int4 cd = S.chunks[own_chunk(i)];
        for (int slot = cd.y + tid; slot < cd.z; slot += BLOCK)
            S.perm[S.cell_start[S.newcell[slot]] + S.rank[slot]] = slot;
    }
    for (int c = s0 + tid; c < s1; c += BLOCK) S.cellcnt[c] = 0;
    if (!grid_sync(bar, gen, S.timeout_ns)) return false;
    // R5: order each cell's particles by id, each cell by the CTA whose own
    // chunk holds the cell's first slot (so the work follows the particles,
    // not the cells, of which dilute replicas have many empty ones); restore
    // the padding-cell counts
    {
        const int32_t *pid = S.pid[set];
        for (int i = 0; i < nloc; ++i) {
            const int4 cd = S.chunks[own_chunk(i)];
            for (int p = cd.y + tid; p < cd.z; p += BLOCK) {
                const int c = S.newcell[S.perm[p]];
                const int a = S.cell_start[c], b = S.cell_start[c + 1];
                if (a != p || b - a < 2) continue;
                for (int j = a + 1; j < b; ++j) {
                    const int pj = S.perm[j];
                    const int key = pid[pj];
                    int k = j - 1;
                    while (k >= a && pid[S.perm[k]] > key) {
                        S.perm[k + 1] = S.perm[k];
                        --k;
                    }
                    S.perm[k + 1] = pj;
                }
            }
        }
        for (int r = blockIdx.x * BLOCK + tid; r < S.nrep; r += gridDim.x * BLOCK) {
            const RepDev &R = S.reps[r];
            S.cellcnt[R.cbase + R.nc * R.nc] = R.cap - R.n;
        }
    }
    if (!grid_sync(bar, gen, S.timeout_ns)) return false;
    // R6: gather into the other set with canonical offsets
    {
        const int ns = set ^ 1;
        V *npos = static_cast<V *>(S.pos[ns][0]);
        V *nvel = static_cast<V *>(S.vel[ns]);
        const V *vel = static_cast<const V *>(S.vel[set]);
        const int32_t *pid = S.pid[set];
        for (int i = 0; i < nloc; ++i) {
            const int4 cd = S.chunks[own_chunk(i)];
            const RepDev &R = S.reps[cd.x];
            const T h = rd<T>(R.h, R.hf);
            const bool canon = mode == RB_ALL;
            for (int slot = cd.y + tid; slot < cd.z; slot += BLOCK) {
                const int old = S.perm[slot];
                V o = pos[old];
                const uint32_t cpk = cell[old];
                const int sx = !canon ? 0 : (o.x >= h ? 1 : (o.x < T(0) ? -1 : 0));
                const int sy = !canon ? 0 : (o.y >= h ? 1 : (o.y < T(0) ? -1 : 0));
                o.x -= (T)sx * h;
                o.y -= (T)sy * h;
                const int ncx = wrap1((int)(cpk & 0xffffu) + sx, R.nc);
                const int ncy = wrap1((int)(cpk >> 16) + sy, R.nc);
                npos[slot] = o;
                nvel[slot] = vel[old];
                S.pid[ns][slot] = pid[old];
                S.cell[ns][slot] = (uint32_t)ncx | ((uint32_t)ncy << 16);
            }
        }
    }
    if (!grid_sync(bar, gen, S.timeout_ns)) return false;
    set ^= 1;
    cur = 0;
    // R7: neighbour lists.  Staged shapes: the chunk windows and lists of
    // the CTA's own chunks in slot order, read only by this CTA, so no
    // barrier follows.  Global-memory shapes: chunks claimed by CTAs, lists
    // in the sorted layout (chunk_lists_sorted); any warp may read them next,
    // so a barrier follows.
    {
        const V *npos = static_cast<const V *>(S.pos[set][0]);
        const uint32_t *ncell = S.cell[set];
        int over = 0;
        if (S.stage) {
            for (int i = tid; i < nloc; i += BLOCK)
                s_desc[i] = make_desc(S, ncell, own_chunk(i), WinParts<T>::value);
            __syncthreads();
            for (int i = 0; i < nloc; ++i)
                for (int slot = s_desc[i].start + tid; slot < s_desc[i].end; slot += BLOCK) {
                    const int cnt = build_list<T>(S, S.reps[s_desc[i].rep], npos, ncell[slot], npos[slot],
                                                  slot, slot);
                    S.nn[slot] = cnt < S.K ? cnt : S.K;
                    over |= cnt > S.K;
                }
        } else {
            for_each_chunk_cta(S, claim0, [&](int c) {
                chunk_lists_sorted<T, BLOCK>(S, set, S.chunks[c], sort_mem, over);
            });
        }
        if (__syncthreads_or(over) && tid == 0) atomicOr(&C->status, (int)DS_NBR_OVERFLOW);
    }
    if (blockIdx.x == 0 && tid == 0) C->n_rebuilds += 1;
    if (!S.stage && !grid_sync(bar, gen, S.timeout_ns)) return false;
    return true;
}

// Flushes the CTA's shared histograms (replica rep, sampling slots in mask)
// to the global block accumulators and clears them.
__device__ __forceinline__ void flush_hist(const SysDev &S, int *sh, int rep, unsigned mask,
                                           const long long *win) {
    const int per = S.n_dx * S.nb;
    for (int k = 0; k < S.n_lg; ++k) {
        if (!(mask >> k & 1u) || win[k] < 0) continue;
        const int blk = (int)((win[k] / S.block_windows) % MD_NBLK);
        for (int e = threadIdx.x; e < per; e += blockDim.x) {
            const int v = sh[k * per + e];
            if (v) {
                const int d = e / S.nb, b = e % S.nb;
                atomicAdd(&S.hist[((((long long)rep * S.n_lg + k) * S.n_dx + d) * MD_NBLK + blk) *
                                      S.nb + b],
                          v);
                sh[k * per + e] = 0;
            }
        }
    }
}

// MDLG sampling of one particle for interval k (Eq. n_i): lattice cells of
// its snapshot and its current position on every lattice, the displacement
// class of each, the continuous displacement moments; the current position
// becomes the snapshot.  bins[d] = -1 when nothing is to be counted.
template <typename T>
__device__ __forceinline__ void sample_particle(const SysDev &S, const RepDev &R, int rep, int k,
                                                bool bin, int id, uint32_t cpk,
                                                typename V2<T>::type on, int *bins, double &m2,
                                                double &m4) {
    using V = typename V2<T>::type;
    uint32_t *scell = S.snap_cell + (long long)k * S.ntot;
    V *soff = static_cast<V *>(S.snap_off) + (long long)k * S.ntot;
    const int cx = (int)(cpk & 0xffffu), cy = (int)(cpk >> 16);
    if (bin) {
        const uint32_t spk = scell[id];
        const V so = soff[id];
        const int scx = (int)(spk & 0xffffu), scy = (int)(spk >> 16);
        int dcx = cx - scx, dcy = cy - scy;
        const int half = R.nc / 2;
        if (dcx > half) dcx -= R.nc; else if (dcx < -half) dcx += R.nc;
        if (dcy > half) dcy -= R.nc; else if (dcy < -half) dcy += R.nc;
        const double ex = (double)dcx * R.h + ((double)on.x - (double)so.x);
        const double ey = (double)dcy * R.h + ((double)on.y - (double)so.y);
        const double ex2 = ex * ex, ey2 = ey * ey;
        m2 = ex2 + ey2;
        m4 = ex2 * ex2 + ey2 * ey2;
        // lattice cells floor(RN(RN(c h + off) / dxl)) mod lx, decided in FP32
        // where that provably gives the same cell (lattice_cell_f32)
        for (int d = 0; d < S.n_dx; ++d) {
            const int lx = R.lx[d];
            const double dxl = R.dxl[d];
            const float invf = R.dxl_invf[d];
            const int ddx = lattice_shift_near(lattice_cell_f32<T>(cx, on.x, R.h, R.hf, dxl, invf, lx) -
                                                   lattice_cell_f32<T>(scx, so.x, R.h, R.hf, dxl, invf, lx),
                                               lx);
            const int ddy = lattice_shift_near(lattice_cell_f32<T>(cy, on.y, R.h, R.hf, dxl, invf, lx) -
                                                   lattice_cell_f32<T>(scy, so.y, R.h, R.hf, dxl, invf, lx),
                                               lx);
            if (ddx >= -S.W && ddx <= S.W && ddy >= -S.W && ddy <= S.W)
                bins[d] = (int)((ddy + S.W) * (2 * S.W + 1) + (ddx + S.W));
            else
                atomicAdd(&S.ovf[((long long)rep * S.n_lg + k) * S.n_dx + d], 1ull);
        }
    }
    scell[id] = cpk;
    soff[id] = on;
}

// Dynamic shared memory of the persistent kernel: sampling histograms,
// chunk descriptors, two staging buffers (window positions, own velocities).
__host__ __device__ inline size_t smem_hist_bytes(int n_lg, int n_dx, int nb) {
    return align16((size_t)n_lg * n_dx * nb * sizeof(int));
}
template <typename T>
__host__ __device__ inline size_t stage_bytes(int chunk) {
    using V = typename V2<T>::type;
    return align16((size_t)WinParts<T>::value * sizeof(V)) + align16((size_t)chunk * sizeof(V)) +
           align16((size_t)(chunk + 4) * sizeof(int32_t)) +
           align16((size_t)chunk * NB_STAGE<T> * sizeof(uint32_t));
}
template <typename T>
__device__ inline Stage<T> stage_at(unsigned char *p, int chunk) {
    using V = typename V2<T>::type;
    Stage<T> B;
    B.pos = reinterpret_cast<V *>(p);
    p += align16((size_t)WinParts<T>::value * sizeof(V));
    B.vel = reinterpret_cast<V *>(p);
    p += align16((size_t)chunk * sizeof(V));
    B.nn = reinterpret_cast<int32_t *>(p);
    p += align16((size_t)(chunk + 4) * sizeof(int32_t));
    B.ent = reinterpret_cast<uint32_t *>(p);
    return B;
}
template <typename T>
__host__ __device__ inline size_t smem_bytes(int n_lg, int n_dx, int nb, int chunk, bool staged) {
    // the two staging buffers exist only when chunks are staged in shared
    // memory; without them more CTAs fit on an SM
    return smem_hist_bytes(n_lg, n_dx, nb) + align16(MAX_CPC * sizeof(ChunkDesc)) +
           (staged ? 2 * stage_bytes<T>(chunk) : sort_scratch_bytes(chunk));
}

// Records the force of one slot by particle id (md_step_forces only).
template <typename T>
__device__ __forceinline__ void debug_force(const SysDev &S, int set, int slot, T fx, T fy) {
    const int id = S.pid[set][slot];
    S.dbg_fx[id] = (double)fx;
    S.dbg_fy[id] = (double)fy;
}

// Velocity-Verlet update of one particle: v += (dt/2m) F twice (the first
// kick completes the previous step unless velocities are at an integer
// step), off += dt v into the other position buffer; tracks the largest
// |v| dt / (skin/2) and non-finite velocities.
template <typename T>
__device__ __forceinline__ void kick_drift(const RepDev &R, typename V2<T>::type oi,
                                           typename V2<T>::type v, T fx, T fy, T hk, T dt,
                                           bool first, float vscale, typename V2<T>::type *pout,
                                           typename V2<T>::type *vel, int slot, float &vm,
                                           bool &bad) {
    // explicit roundings (no contraction), so that every call site gives the
    // same bits (FMA contraction would otherwise be decided per call site)
    if (!first) {
        v.x = axpyT(v.x, hk, fx);
        v.y = axpyT(v.y, hk, fy);
    }
    v.x = axpyT(v.x, hk, fx);
    v.y = axpyT(v.y, hk, fy);
    typename V2<T>::type on;
    on.x = axpyT(oi.x, dt, v.x);
    on.y = axpyT(oi.y, dt, v.y);
    pout[slot] = on;
    vel[slot] = v;
    const float vx = (float)v.x, vy = (float)v.y;
    const float sp = __fmul_rn(sqrtf(__fmaf_rn(vx, vx, __fmul_rn(vy, vy))), vscale);
    vm = fmaxf(vm, sp);
    bad |= !(sp < 1e30f);   // non-finite velocity
}

// ---------------------------------------------------------------- persistent step kernel
// Advances all replicas by nsteps velocity-Verlet steps (Sec. 4).  Per step:
//   force pass -- per slot: force F_s from the neighbour list; v += (dt/2m) F
//     twice (the first kick completes the previous step unless velocities are
//     at an integer step); off += dt v into the other position buffer; the
//     largest |v| dt of the step is reduced grid-wide;
//   grid barrier; every CTA adds it to the same displacement bound;
//   sampling pass (steps t = n_equil + m*lg_every[k] only) -- bin each new
//     position against its snapshot (Eq. n_i) and replace the snapshot;
//   rebuild (canonical cells, cell list + neighbour lists) once the
//     accumulated bound on displacements since the last rebuild reaches half
//     the skin: until then no pair can have come within rc without being
//     listed.  One bound for the batch, so every replica is rebuilt together
//     (one sort, six or seven grid barriers); for a single replica this is the rule
//     of the resident engine, which keeps one bound per replica.
// CTAs per SM the register allocation is sized for: half occupancy (64
// registers), or with DENSE full occupancy (32 registers: the spills cost
// less than the extra latency hiding gains on large ensembles, whose
// neighbour gathers also use the L1 left free when chunks are not staged;
// small systems prefer the former).  The autotuner chooses.
constexpr int md_min_ctas(int block, bool dense) { return (dense ? 2048 : 1024) / block; }

template <typename T, int BLOCK, bool DENSE>
__global__ void __launch_bounds__(BLOCK, md_min_ctas(BLOCK, DENSE)) k_md_persistent(SysDev S, long long step0,
                                                                           long long nsteps,
                                                                           int phase_half,
                                                                           int force_rebuild) {
    using V = typename V2<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int chunk = S.ppt * BLOCK;
    const size_t hb = smem_hist_bytes(S.n_lg, S.n_dx, S.nb);
    int *sh_hist = reinterpret_cast<int *>(smem);
    ChunkDesc *s_desc = reinterpret_cast<ChunkDesc *>(smem + hb);
    unsigned char *stg = smem + hb + align16(MAX_CPC * sizeof(ChunkDesc));
    const Stage<T> B0 = stage_at<T>(stg, chunk), B1 = stage_at<T>(stg + stage_bytes<T>(chunk), chunk);
    __shared__ unsigned s_due;
    __shared__ long long s_win[MD_MAX_LG];
    __shared__ float s_vmax[BLOCK / 32];
    __shared__ double s_dmax[BLOCK / 32];
    Control *C = S.ctl;
    const GridBarrier bar{&C->bar_count, &C->bar_gen, &C->status};
    const int tid = threadIdx.x, lane = tid & 31;
    unsigned gen = 0;
    if (tid == 0) gen = ld_acquire_gpu(&C->bar_gen);
    int set = C->set, cur = C->cur;
    const int nloc = own_chunks(S.nchunks);
    unsigned long long claim0 = 0;   // claim counter at the start of the next claiming pass
    const int per_lg = S.n_dx * S.nb;
    for (int e = tid; e < S.n_lg * per_lg; e += BLOCK) sh_hist[e] = 0;
    // one bound for the whole batch: the largest of the replicas' bounds (a
    // resident launch may have left them different)
    double disp = 0.0;
    {
        double m = 0.0;
        for (int r = tid; r < S.nrep; r += BLOCK) m = fmax(m, S.disp_rep[r]);
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_dmax[tid >> 5] = m;
        __syncthreads();
        for (int w = 0; w < BLOCK / 32; ++w) disp = fmax(disp, s_dmax[w]);
    }

    if (force_rebuild) {
        // RB_ALL: canonical cells (a new state); RB_NONE: sort and lists of a
        // state written in another order, no particle's cell moved
        if (!rebuild<T, BLOCK>(S, set, cur, gen, nloc, s_desc, force_rebuild, claim0, stg)) return;
        if (force_rebuild == RB_ALL) disp = 0.0;
    } else {
        for (int i = tid; i < nloc; i += BLOCK)
            s_desc[i] = make_desc(S, S.cell[set], own_chunk(i), WinParts<T>::value);
    }
    __syncthreads();
    for (long long it = 0; it < nsteps; ++it) {
        const long long s = step0 + it;
        if (tid == 0) {
            unsigned due = 0;
            const long long t = s + 1 - S.n_equil;
            for (int k = 0; k < S.n_lg; ++k) {
                if (t >= 0 && t % S.lg_every[k] == 0) {
                    due |= 1u << k;
                    s_win[k] = t / S.lg_every[k] - 1;   // -1: first snapshot only
                } else {
                    s_win[k] = -1;
                }
            }
            s_due = due;
            if (blockIdx.x == 0) C->vmax[(s + 1) % 3] = 0u;
        }
        const bool first = (it == 0) ? (phase_half == 0) : false;
        const V *pin = static_cast<const V *>(S.pos[set][cur]);
        V *pout = static_cast<V *>(S.pos[set][cur ^ 1]);
        V *vel = static_cast<V *>(S.vel[set]);
        float vm = 0.0f;   // largest |v| dt / (skin/2) of this CTA's particles
        bool bad = false;
        // ---- force pass
        if (S.stage) {
            // chunk i+1 is staged in shared memory while chunk i is computed
            if (nloc > 0) stage_chunk<T, BLOCK>(S, S.reps[s_desc[0].rep], s_desc[0], pin, vel, B0);
            cp_async_commit();
            for (int i = 0; i < nloc; ++i) {
                const bool odd = i & 1;
                if (i + 1 < nloc)
                    stage_chunk<T, BLOCK>(S, S.reps[s_desc[i + 1].rep], s_desc[i + 1], pin, vel,
                                          odd ? B0 : B1);
                cp_async_commit();
                cp_async_wait<1>();
                __syncthreads();
                const ChunkDesc d = s_desc[i];
                const RepDev &R = S.reps[d.rep];
                const Stage<T> &B = odd ? B1 : B0;
                const T hk = rd<T>(R.hk, R.hkf), dt = rd<T>(R.dt, R.dtf);
                const float vscale = (float)(R.dt / R.half_skin);
                for (int li = tid; li < d.end - d.start; li += BLOCK) {
                    const int slot = d.start + li;
                    const int ks = d.ok ? window_index(d, R, slot) : -1;
                    const V oi = ks >= 0 ? B.pos[ks] : pin[slot];
                    T fx = T(0), fy = T(0);
                    lj_list<T>(S, R, d, B.pos, B.ent + (li >> 5) * NB_STAGE<T> * 32 + (li & 31), pin,
                               oi, slot, B.nn[li], fx, fy);
                    if (S.dbg_fx && it == nsteps - 1) debug_force(S, set, slot, fx, fy);
                    kick_drift<T>(R, oi, B.vel[li], fx, fy, hk, dt, first, vscale, pout, vel, slot, vm,
                                  bad);
                }
                __syncthreads();   // this buffer is refilled for chunk i+2
            }
            cp_async_wait<0>();
        } else {
            // neighbours straight from global memory (L1/L2); groups from the
            // dynamic distribution (for_each_group)
            const ChunkDesc none{};
            for_each_group<BLOCK>(S, claim0, [&](const int4 &cd, int g0) {
                // sorted layout: position q holds the list and count of the
                // slot its count word names; the first list batch is read
                // with the count, the slot's state once it arrives
                const int q = g0 + lane;
                if (q >= cd.z) return;
                uint32_t e[NB_STAGE<T>];
                const uint32_t *lst = S.nbr + (long long)(q >> 5) * S.K * 32 + (q & 31);
#pragma unroll
                for (int u = 0; u < NB_STAGE<T>; ++u) e[u] = lst[u * 32];
                const int w = S.nn[q];
                const int slot = cd.y + (w >> 16);
                const RepDev &R = S.reps[cd.x];
                const V oi = pin[slot];
                T fx = T(0), fy = T(0);
                lj_list_from<T>(S, R, none, nullptr, pin, oi, q, w & 0xffff, e, fx, fy);
                // the velocity and the kick's constants only now: fewer values
                // live in the pair loop of the 32-register budget (measured:
                // faster than requesting the velocity before the sum)
                const V vi = vel[slot];
                const T hk = rd<T>(R.hk, R.hkf), dt = rd<T>(R.dt, R.dtf);
                const float vscale = (float)(R.dt / R.half_skin);
                if (S.dbg_fx && it == nsteps - 1) debug_force(S, set, slot, fx, fy);
                kick_drift<T>(R, oi, vi, fx, fy, hk, dt, first, vscale, pout, vel, slot, vm, bad);
            });
        }
        for (int o = 16; o > 0; o >>= 1) vm = fmaxf(vm, __shfl_xor_sync(0xffffffffu, vm, o));
        if (lane == 0) s_vmax[tid >> 5] = vm;
        if (__syncthreads_or(bad) && tid == 0) atomicOr(&C->status, (int)DS_NONFINITE);
        if (tid == 0) {
            float m = 0.0f;
            for (int w = 0; w < BLOCK / 32; ++w) m = fmaxf(m, s_vmax[w]);
            atomicMax(&C->vmax[s % 3], __float_as_uint(m));   // non-negative floats order as uints
        }
        // the barrier self-test: one CTA never arrives, so the others' wait
        // runs into its limit (nothing else is skipped; the CTA returns)
        if (it == 0 && S.dbg_leave_cta == (int)blockIdx.x) return;
        if (!grid_sync(bar, gen, S.timeout_ns)) return;
        cur ^= 1;
        // every CTA accumulates the same bound, in units of half the skin
        disp += (double)__uint_as_float(*(volatile unsigned *)&C->vmax[s % 3]) * 1.0000001;
        // ---- sampling pass
        const unsigned due = s_due;
        if (due) {
            const V *pnow = static_cast<const V *>(S.pos[set][cur]);
            const int32_t *pid = S.pid[set];
            const uint32_t *cell = S.cell[set];
            int hist_rep = -1;
            for (int i = 0; i < nloc; ++i) {
                const int4 cd = S.chunks[own_chunk(i)];
                const RepDev &R = S.reps[cd.x];
                if (cd.x != hist_rep) {
                    if (hist_rep >= 0) {
                        __syncthreads();
                        flush_hist(S, sh_hist, hist_rep, due, s_win);
                        __syncthreads();
                    }
                    hist_rep = cd.x;
                }
                for (int base = cd.y; base < cd.z; base += BLOCK) {
                    const int slot = base + tid;
                    const bool active = slot < cd.z;
                    int id = 0;
                    uint32_t cpk = 0;
                    V on{};
                    if (active) {
                        id = pid[slot];
                        cpk = cell[slot];
                        on = pnow[slot];
                    }
                    for (int k = 0; k < S.n_lg; ++k) {
                        if (!(due >> k & 1u)) continue;
                        const bool bin = s_win[k] >= 0;
                        int bins[MD_MAX_DX] = {-1, -1, -1, -1};
                        double m2 = 0.0, m4 = 0.0;
                        if (active) sample_particle<T>(S, R, cd.x, k, bin, id, cpk, on, bins, m2, m4);
                        if (bin) {
                            for (int d = 0; d < S.n_dx; ++d)
                                warp_hist_add(sh_hist + k * per_lg + d * S.nb, bins[d], lane);
                            for (int o = 16; o > 0; o >>= 1) {
                                m2 += __shfl_xor_sync(0xffffffffu, m2, o);
                                m4 += __shfl_xor_sync(0xffffffffu, m4, o);
                            }
                            if (lane == 0 && (base + (tid & ~31)) < cd.z) {
                                double *mp = S.mom + ((long long)(slot >> 5) * S.n_lg + k) * 2;
                                mp[0] += m2;
                                mp[1] += m4;
                            }
                        }
                    }
                }
            }
            if (hist_rep >= 0) {
                __syncthreads();
                flush_hist(S, sh_hist, hist_rep, due, s_win);
            }
        }
        if (disp >= 1.0) {
            if (!rebuild<T, BLOCK>(S, set, cur, gen, nloc, s_desc, RB_ALL, claim0, stg)) return;
            disp = 0.0;
        }
        __syncthreads();   // s_due / s_win / s_vmax are rewritten in the next step
    }
    if (blockIdx.x == 0) {
        // every replica's bound is the batch's (a sort that moved nothing
        // keeps the replicas' own bounds)
        if (nsteps > 0 || force_rebuild == RB_ALL)
            for (int r = tid; r < S.nrep; r += BLOCK) S.disp_rep[r] = disp;
        if (tid == 0) {
            C->set = set;
            C->cur = cur;
        }
    }
}

// ---------------------------------------------------------------- observation kernel
// One pass at the current step without moving particles: forces, optional
// completion of the half kick (velocities then refer to the current step),
// per-warp energy/momentum partials, outputs in particle-id order, and
// snapshots for the sampling slots in snap_mask.
struct ObsArgs {
    int complete;          // apply v += (dt/2m) F (velocities were half-step)
    double *epart;         // [nslots/32][4] KE, PE, Px, Py or NULL
    double *fx, *fy, *fabs_sum;   // by particle id, or NULL
    double *x, *y, *vx, *vy;      // by particle id, or NULL
    int32_t *raw_cell;             // by particle id, or NULL (linear cy*nc+cx)
    void *raw_x, *raw_y;
    unsigned snap_mask;            // sampling slots whose snapshot is taken now
};

template <typename T>
__global__ void k_observe(SysDev S, ObsArgs A) {
    using V = typename V2<T>::type;
    const int set = S.ctl->set, cur = S.ctl->cur;
    const V *pos = static_cast<const V *>(S.pos[set][cur]);
    V *vel = static_cast<V *>(S.vel[set]);
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0, pe = 0.0, px = 0.0, py = 0.0;
    if (slot < S.nslots) {
        const RepDev &R = S.reps[S.gran_rep[slot / GRAN]];
        if (slot < R.pbase + R.n) {
            const V oi = pos[slot];
            const uint32_t cpk = S.cell[set][slot];
            V v = vel[slot];
            T fx = T(0), fy = T(0);
            double fa = 0.0;
            // forces only for the outputs that use them (the half kick, the
            // force readout, the potential energy); a snapshot or state
            // readout needs none
            if (A.complete || A.fx || A.epart)
                lj_stencil<T, true>(R, pos, S.cell_start, cpk, oi, slot, fx, fy, pe, fa);
            if (A.complete) {
                const T hk = rd<T>(R.hk, R.hkf);
                v.x = axpyT(v.x, hk, fx);
                v.y = axpyT(v.y, hk, fy);
                vel[slot] = v;
            }
            ke = 0.5 * R.mass * ((double)v.x * (double)v.x + (double)v.y * (double)v.y);
            px = R.mass * (double)v.x;
            py = R.mass * (double)v.y;
            const int id = S.pid[set][slot];
            if (A.fx) {
                A.fx[id] = (double)fx;
                A.fy[id] = (double)fy;
                if (A.fabs_sum) A.fabs_sum[id] = fa;
            }
            const int cx = (int)(cpk & 0xffffu), cy = (int)(cpk >> 16);
            if (A.x) {
                double X = cell_position(cx, R.h, (double)oi.x);
                double Y = cell_position(cy, R.h, (double)oi.y);
                X -= R.L * floor(X / R.L);
                Y -= R.L * floor(Y / R.L);
                if (X >= R.L) X -= R.L;
                if (Y >= R.L) Y -= R.L;
                A.x[id] = X;
                A.y[id] = Y;
                A.vx[id] = (double)v.x;
                A.vy[id] = (double)v.y;
            }
            if (A.raw_cell) {
                A.raw_cell[id] = cy * R.nc + cx;
                static_cast<T *>(A.raw_x)[id] = oi.x;
                static_cast<T *>(A.raw_y)[id] = oi.y;
            }
            for (int k = 0; k < S.n_lg; ++k) {
                if (!(A.snap_mask >> k & 1u)) continue;
                S.snap_cell[(long long)k * S.ntot + id] = cpk;
                static_cast<V *>(S.snap_off)[(long long)k * S.ntot + id] = oi;
            }
        }
    }
    if (A.epart) {
        for (int o = 16; o > 0; o >>= 1) {
            ke += __shfl_xor_sync(0xffffffffu, ke, o);
            pe += __shfl_xor_sync(0xffffffffu, pe, o);
            px += __shfl_xor_sync(0xffffffffu, px, o);
            py += __shfl_xor_sync(0xffffffffu, py, o);
        }
        if ((threadIdx.x & 31) == 0 && slot < S.nslots) {
            double *e = A.epart + (long long)(slot >> 5) * 4;
            e[0] = ke;
            e[1] = pe;
            e[2] = px;
            e[3] = py;
        }
    }
}

}  // namespace mdlg
