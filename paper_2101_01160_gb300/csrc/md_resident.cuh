// The shared-memory-resident engine of the batched FP32 ensemble (Sec. 4 MD
// with the Sec. 2 sampling fused), an alternative to k_md_persistent for
// md_step.  Included by md.cu only.
//
// Each replica is cut into g horizontal slabs of whole MD-cell rows; each
// slab lives in the shared memory of one CTA for the whole launch: offsets
// (double buffered), velocities, cells, ids and the Verlet neighbour lists.
// A step reads nothing from global memory but the two boundary rows of the
// neighbouring slabs (the halo, 8 bytes per particle, through L2) and the
// sampling snapshots once per window.  The g CTAs of a replica (its gang)
// meet at one bounded barrier per step; replicas never wait for each other,
// and a replica with g = 1 waits for nobody.  A host plan deals the slabs of
// all replicas to the CTAs of one cooperative launch (one CTA per SM) by
// list scheduling; each CTA runs its slabs one after another.
//
// Every replica's trajectory equals, bit for bit, the one k_md_persistent
// gives that replica alone: the rebuild rule is per replica (canonical cells
// once the replica's displacement bound reaches half the skin -- the global
// engine's rule for a single replica; for a batch it rebuilds all replicas
// together), the canonicalisation and kick/drift arithmetic are the same,
// and each particle's force is summed over the same pairs in the same order
// -- the 3x3 stencil of its cell row by row, column by column, by id inside
// a cell (the lists are built in that order; pairs beyond rc add nothing,
// so when a list was built does not matter).  So a replica's results do not
// depend on the batch, the slab plan or how md_step calls are split; only
// the FP64 moment partial sums are grouped per slab.
#pragma once

#include "md_kernels.cuh"

namespace mdlg {

constexpr int RES_THREADS = 1024;
constexpr int RES_CTAS_PER_SM = 1;   // row slabs of wide dense replicas need a whole SM's shared memory
constexpr int RES_NCC = 2048;      // coarse cells of the list-building grid
constexpr int RES_PCAP = 8192;     // own particles of one slab (index + 2 halo < 2^14)
constexpr int RES_MAXLIST = 255;   // neighbours of one particle (u8 row counts)
// steps per launch: a longer md_step is split, so that no CTA waits at a
// slab's first barrier for longer than its gang members' earlier slabs
// take over this many steps (far below the barrier's time limit)
constexpr long long RES_MAX_STEPS = 2000;

// One slab: replica rep cut into g slabs, this is slab k, MD-cell rows
// [r0, r1); slab k' of the replica runs on CTA cta0 + k'.
struct ResJob {
    int32_t rep, g, k, r0, r1, p_cap, h_cap, cta0;
};

struct ResDev {
    const ResJob *jobs;       // grouped by CTA, in execution order
    const int32_t *job_start; // [grid + 1]
    float2 *halo_off;         // [grid][2 sides][2 parities][hmax]: boundary offsets
    uint2 *halo_ci;           // [grid][2 sides][hmax]: boundary cell, id
    int32_t *halo_n;          // [grid][2]
    float4 *mig_a;            // [grid][2 directions][hmax]: offset, velocity
    uint2 *mig_b;             // [grid][2 directions][hmax]: cell, id
    int32_t *mig_n;           // [grid][2]
    int32_t *slab_n;          // [grid]: particles of the slab at write-back
    unsigned *gbar;           // [nrep][2]: gang barrier arrivals, generation
    unsigned long long *job_ns;   // [jobs]: each slab's time from its first barrier to its store
    int32_t hmax;
    int32_t smem_bytes;       // dynamic shared memory of the launch
};

// ---------------------------------------------------------------- helpers
// Exclusive prefix sum of v over the CTA in thread order; *total receives
// the sum.  All threads call it.  s_w: 33 ints of shared scratch.
__device__ __forceinline__ int block_excl_scan(int v, int *s_w, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    __syncthreads();
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int y = lane < nw ? s_w[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) s_w[lane] = y;   // inclusive warp totals
        if (lane == 31) s_w[32] = y;
    }
    __syncthreads();
    const int before = (w ? s_w[w - 1] : 0) + x - v;
    *total = s_w[32];
    __syncthreads();
    return before;
}

// Barrier of the g CTAs of one replica, with a bounded wait (limit_ns): a
// CTA that waits longer sets DS_TIMEOUT.  Returns false once a failure that
// stops the launch has been flagged (timeout or capacity), so that the gang
// leaves instead of waiting.  my_gen: the generation thread 0 last saw.
__device__ __forceinline__ bool gang_sync(unsigned *bar, int g, unsigned &my_gen, int *status,
                                          uint64_t limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (g > 1) {
            const unsigned gv = my_gen;
            __threadfence();
            const unsigned old = atom_add_acqrel_gpu(&bar[0], 1u);
            if (old == (unsigned)g - 1u) {
                atomicExch(&bar[0], 0u);
                st_release_gpu(&bar[1], gv + 1u);
            } else {
                const uint64_t t0 = global_ns();
                unsigned spins = 0;
                while (ld_acquire_gpu(&bar[1]) == gv) {
                    if ((++spins & 63u) == 0) {
                        if ((*(volatile int *)status) & (DS_TIMEOUT | DS_CAPACITY)) break;
                        if (global_ns() - t0 > limit_ns) {
                            atomicOr(status, (int)DS_TIMEOUT);
                            break;
                        }
                    }
                    __nanosleep(20);
                }
            }
            my_gen = gv + 1u;
            __threadfence();
        }
        s_ok = ((*(volatile int *)status) & (DS_TIMEOUT | DS_CAPACITY)) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void res_fail(int *status, int flag) { atomicOr(status, flag); }

// Shared-memory layout of one slab.  Own particles occupy indices [0, p_cap)
// and the halo [p_cap, p_cap + 2 h_cap) (upper halo first) of the cell and
// id arrays and of list entries; own offsets are double buffered (a step
// reads one and writes the other), halo offsets single (rewritten after the
// step's barrier, when every read of them is done).  The coarse-grid
// scratch of a list build lives in the spare own-offset buffer.  A list
// entry is the neighbour's index | (dcx + 1) << 14; a particle's entries are
// in stencil order, rows dcy = -1, 0, 1 ending at lst + the two counts in
// rend and at the next particle's start.
// The dynamic shared memory of k_md_resident.  Slab arrays are addressed as
// byte offsets into it, so that every access compiles to a shared-memory
// load or store with 32-bit addresses.
extern __shared__ __align__(16) unsigned char res_smem[];

struct Slab {
    uint32_t o_off[2], o_hoff, o_vel, o_cell, o_id, o_lst, o_rend, o_bidx, o_bpos, o_ent;
    int e_cap;
    __device__ __forceinline__ float2 *off(int b) const { return reinterpret_cast<float2 *>(res_smem + o_off[b]); }
    __device__ __forceinline__ float2 *hoff() const { return reinterpret_cast<float2 *>(res_smem + o_hoff); }
    __device__ __forceinline__ float2 *vel() const { return reinterpret_cast<float2 *>(res_smem + o_vel); }
    __device__ __forceinline__ uint32_t *cell() const { return reinterpret_cast<uint32_t *>(res_smem + o_cell); }
    __device__ __forceinline__ int32_t *id() const { return reinterpret_cast<int32_t *>(res_smem + o_id); }
    __device__ __forceinline__ uint32_t *lst() const { return reinterpret_cast<uint32_t *>(res_smem + o_lst); }
    __device__ __forceinline__ uint16_t *rend() const { return reinterpret_cast<uint16_t *>(res_smem + o_rend); }
    __device__ __forceinline__ uint16_t *bidx() const { return reinterpret_cast<uint16_t *>(res_smem + o_bidx); }
    // per own particle: side << 15 | position in that side's boundary set, or
    // RES_NOB (not in the first or the last row)
    __device__ __forceinline__ uint16_t *bpos() const { return reinterpret_cast<uint16_t *>(res_smem + o_bpos); }
    __device__ __forceinline__ uint16_t *ent() const { return reinterpret_cast<uint16_t *>(res_smem + o_ent); }
    // build scratch in the spare own-offset buffer of cur
    __device__ __forceinline__ unsigned char *scratch(int cur) const { return res_smem + o_off[cur ^ 1]; }
};

constexpr uint32_t RES_IDX = (1u << 14) - 1u;
constexpr uint16_t RES_NOB = 0xffffu;

__host__ __device__ inline size_t res_off_bytes(int p_cap, int h_cap) {
    // an own-offset buffer, large enough to hold the build scratch
    const size_t scratch = align16(((size_t)p_cap + 2 * (size_t)h_cap) * sizeof(uint16_t)) +
                           align16((RES_NCC + 1) * sizeof(int32_t));
    const size_t own = align16((size_t)p_cap * sizeof(float2));
    return own > scratch ? own : scratch;
}

__host__ __device__ inline size_t res_slab_bytes(int p_cap, int h_cap, int e_cap) {
    const size_t ph = (size_t)p_cap + 2 * (size_t)h_cap;
    return 2 * res_off_bytes(p_cap, h_cap) + align16(2 * (size_t)h_cap * sizeof(float2)) +
           align16((size_t)p_cap * sizeof(float2)) + align16(ph * sizeof(uint32_t)) +
           align16(ph * sizeof(int32_t)) + align16(((size_t)p_cap + 1) * sizeof(uint32_t)) +
           align16((size_t)p_cap * sizeof(uint16_t)) + align16(2 * (size_t)h_cap * sizeof(uint16_t)) +
           align16((size_t)p_cap * sizeof(uint16_t)) + align16((size_t)e_cap * sizeof(uint16_t));
}

__device__ inline Slab res_layout(uint32_t base, int p_cap, int h_cap, size_t avail) {
    Slab L;
    const size_t ph = (size_t)p_cap + 2 * (size_t)h_cap;
    uint32_t p = base;
    const uint32_t ob = (uint32_t)res_off_bytes(p_cap, h_cap);
    L.o_off[0] = p; p += ob;
    L.o_off[1] = p; p += ob;
    L.o_hoff = p; p += (uint32_t)align16(2 * (size_t)h_cap * sizeof(float2));
    L.o_vel = p; p += (uint32_t)align16((size_t)p_cap * sizeof(float2));
    L.o_cell = p; p += (uint32_t)align16(ph * sizeof(uint32_t));
    L.o_id = p; p += (uint32_t)align16(ph * sizeof(int32_t));
    L.o_lst = p; p += (uint32_t)align16(((size_t)p_cap + 1) * sizeof(uint32_t));
    L.o_rend = p; p += (uint32_t)align16((size_t)p_cap * sizeof(uint16_t));
    L.o_bidx = p; p += (uint32_t)align16(2 * (size_t)h_cap * sizeof(uint16_t));
    L.o_bpos = p; p += (uint32_t)align16((size_t)p_cap * sizeof(uint16_t));
    L.o_ent = p;
    const size_t used = (size_t)(p - base);
    L.e_cap = used < avail ? (int)((avail - used) / sizeof(uint16_t)) : 0;
    return L;
}

// Offset of own or halo particle j in the buffer holding the current
// positions.
__device__ __forceinline__ float2 res_off(const Slab &L, int cur, int p_cap, int j) {
    return j < p_cap ? L.off(cur)[j] : L.hoff()[j - p_cap];
}

// State of the slab a CTA is running.
struct SlabRun {
    ResJob J;
    int p;          // own particles
    int nh[2];      // upper / lower halo particles
    int nb[2];      // own particles of the first / last row
    int cur;        // offset buffer holding the current positions
    int par;        // parity of the global halo buffers holding them
    int up, down;   // CTAs of the neighbouring slabs
};

__device__ __forceinline__ int res_relrow(const SlabRun &X, int nc, int cy) {
    if (X.J.g == 1) return cy;
    int r = cy - X.J.r0 + 1;
    if (r < 0) r += nc;
    else if (r >= nc) r -= nc;
    return r;
}

// ---------------------------------------------------------------- slab load / store
// Collects the replica's particles whose cell row lies in the slab, in slot
// order, from the global state (set, buffer cur).
__device__ bool res_load(const SysDev &S, const RepDev &R, const Slab &L, SlabRun &X, int set, int gcur,
                         int *s_w) {
    const float2 *pos = static_cast<const float2 *>(S.pos[set][gcur]);
    const float2 *vel = static_cast<const float2 *>(S.vel[set]);
    const uint32_t *cell = S.cell[set];
    const int32_t *pid = S.pid[set];
    int p = 0;
    bool over = false;
    for (int base = R.pbase; base < R.pbase + R.n; base += RES_THREADS) {
        const int slot = base + (int)threadIdx.x;
        int f = 0;
        uint32_t c = 0;
        if (slot < R.pbase + R.n) {
            c = cell[slot];
            const int cy = (int)(c >> 16);
            f = X.J.g == 1 || (cy >= X.J.r0 && cy < X.J.r1);
        }
        int tot;
        const int at = p + block_excl_scan(f, s_w, &tot);
        if (f) {
            if (at < X.J.p_cap) {
                L.off(X.cur)[at] = pos[slot];
                L.vel()[at] = vel[slot];
                L.cell()[at] = c;
                L.id()[at] = pid[slot];
            } else {
                over = true;
            }
        }
        p += tot;
    }
    X.p = p;
    return !__syncthreads_or(over) && p <= X.J.p_cap;
}

// Writes the slab back into the other set of the global state, the slabs of
// the replica one after another (slab k after the particles of slabs < k).
__device__ bool res_store(const SysDev &S, const ResDev &D, const RepDev &R, const Slab &L, const SlabRun &X,
                          int nset, unsigned &my_gen, unsigned *bar) {
    __shared__ int s_off;
    if (threadIdx.x == 0) D.slab_n[blockIdx.x] = X.p;
    if (!gang_sync(bar, X.J.g, my_gen, &S.ctl->status, S.timeout_ns)) return false;
    if (threadIdx.x == 0) {
        int o = 0;
        for (int k = 0; k < X.J.k; ++k) o += *(volatile int *)&D.slab_n[X.J.cta0 + k];
        s_off = o;
        if (o + X.p > R.n) res_fail(&S.ctl->status, DS_CAPACITY);   // cannot happen: particles are conserved
    }
    __syncthreads();
    if (s_off + X.p > R.n) return false;
    float2 *pos = static_cast<float2 *>(S.pos[nset][0]);
    float2 *vel = static_cast<float2 *>(S.vel[nset]);
    const int b = R.pbase + s_off;
    for (int i = threadIdx.x; i < X.p; i += RES_THREADS) {
        pos[b + i] = L.off(X.cur)[i];
        vel[b + i] = L.vel()[i];
        S.cell[nset][b + i] = L.cell()[i];
        S.pid[nset][b + i] = L.id()[i];
    }
    // the next job may reuse slab_n only after every gang member read it
    return gang_sync(bar, X.J.g, my_gen, &S.ctl->status, S.timeout_ns);
}

// ---------------------------------------------------------------- halo
// Publishes the first and last rows (cells, ids and current offsets) and
// collects the neighbours' into the halo: the upper halo is the up
// neighbour's first row, the lower halo the down neighbour's last row.
__device__ bool res_halo_full(const SysDev &S, const ResDev &D, const RepDev &R, const Slab &L, SlabRun &X,
                              unsigned &my_gen, unsigned *bar, int *s_w) {
    if (X.J.g == 1) {
        X.nh[0] = X.nh[1] = 0;
        return true;
    }
    const int me = blockIdx.x;
    const int rows[2] = {X.J.r0, X.J.r1 - 1};
    bool over = false;
    for (int i = threadIdx.x; i < X.p; i += RES_THREADS) L.bpos()[i] = RES_NOB;
    __syncthreads();
    for (int side = 0; side < 2; ++side) {
        int n = 0;
        for (int base = 0; base < X.p; base += RES_THREADS) {
            const int i = base + (int)threadIdx.x;
            const int f = i < X.p && (int)(L.cell()[i] >> 16) == rows[side];
            int tot;
            const int at = n + block_excl_scan(f, s_w, &tot);
            if (f) {
                if (at < X.J.h_cap) {
                    L.bidx()[side * X.J.h_cap + at] = (uint16_t)i;
                    L.bpos()[i] = (uint16_t)((side << 15) | at);
                    const long long gi = ((long long)me * 2 + side) * D.hmax + at;
                    D.halo_ci[gi] = make_uint2(L.cell()[i], (uint32_t)L.id()[i]);
                    D.halo_off[(((long long)me * 2 + side) * 2 + X.par) * D.hmax + at] = L.off(X.cur)[i];
                } else {
                    over = true;
                }
            }
            n += tot;
        }
        X.nb[side] = min(n, X.J.h_cap);
        if (threadIdx.x == 0) D.halo_n[me * 2 + side] = n;
    }
    if (__syncthreads_or(over)) res_fail(&S.ctl->status, DS_CAPACITY);
    if (!gang_sync(bar, X.J.g, my_gen, &S.ctl->status, S.timeout_ns)) return false;
    // upper halo <- up neighbour's first row (side 0); lower <- down's last (side 1)
    const int src[2] = {X.up, X.down};
    for (int h = 0; h < 2; ++h) {
        const int side = h == 0 ? 0 : 1;
        const int n = *(volatile int *)&D.halo_n[src[h] * 2 + side];
        if (n > X.J.h_cap) {
            res_fail(&S.ctl->status, DS_CAPACITY);
            return false;
        }
        X.nh[h] = n;
        const int o = X.J.p_cap + h * X.J.h_cap;
        for (int i = threadIdx.x; i < n; i += RES_THREADS) {
            const uint2 ci = D.halo_ci[((long long)src[h] * 2 + side) * D.hmax + i];
            L.cell()[o + i] = ci.x;
            L.id()[o + i] = (int32_t)ci.y;
            L.hoff()[h * X.J.h_cap + i] = D.halo_off[(((long long)src[h] * 2 + side) * 2 + X.par) * D.hmax + i];
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- lists
// Neighbour lists of the own particles: every particle within rv in the 3x3
// stencil of its cell, in stencil order (rows dy = -1, 0, 1, in each row
// columns dx = -1, 0, 1) and by id inside a cell -- the order of build_list
// and lj_stencil.  Candidates are found through a coarse grid (rows of MD
// cells x columns of cw MD cells, at most RES_NCC cells) whose members are
// sorted by (column, id); the grid lives in the spare offset buffer.
__device__ bool res_lists(const SysDev &S, const RepDev &R, const Slab &L, const SlabRun &X, int *s_w) {
    const int nc = R.nc;
    const int G = X.J.g == 1 ? nc : (X.J.r1 - X.J.r0) + 2;   // <= RES_NCC (plan)
    const int ncolmax = RES_NCC / G;
    const int cw = (nc + ncolmax - 1) / ncolmax;
    const int ncol = (nc + cw - 1) / cw;                    // G * ncol <= RES_NCC
    const int ncells = G * ncol;
    const int pc = X.J.p_cap;
    const int ph = pc + 2 * X.J.h_cap;
    unsigned char *scr = L.scratch(X.cur);
    uint16_t *mem = reinterpret_cast<uint16_t *>(scr);
    int32_t *ccs = reinterpret_cast<int32_t *>(scr + align16((size_t)ph * sizeof(uint16_t)));
    auto member = [&](int j) {   // own or filled halo slot
        return j < X.p || (j >= pc && j < pc + X.nh[0]) ||
               (j >= pc + X.J.h_cap && j < pc + X.J.h_cap + X.nh[1]);
    };
    auto ccell = [&](uint32_t c) {   // -1 for a row outside the grid (cannot happen)
        const int cx = (int)(c & 0xffffu), cy = (int)(c >> 16);
        const int r = res_relrow(X, nc, cy);
        return (r < 0 || r >= G || cx >= nc) ? -1 : r * ncol + cx / cw;
    };
    // counting sort of own and halo particles by coarse cell (inclusive sum,
    // then a decrementing scatter leaves ccs[c] = first member of c)
    for (int c = threadIdx.x; c <= ncells; c += RES_THREADS) ccs[c] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < ph; j += RES_THREADS) {
        const int c = member(j) ? ccell(L.cell()[j]) : -1;
        if (c >= 0) atomicAdd(&ccs[c], 1);
    }
    __syncthreads();
    {
        int carry = 0;
        for (int c0 = 0; c0 < ncells; c0 += RES_THREADS) {
            const int c = c0 + (int)threadIdx.x;
            const int v = c < ncells ? ccs[c] : 0;
            int tot;
            const int ex = block_excl_scan(v, s_w, &tot);
            if (c < ncells) ccs[c] = carry + ex + v;
            carry += tot;
        }
        if (threadIdx.x == 0) ccs[ncells] = carry;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < ph; j += RES_THREADS) {
        const int c = member(j) ? ccell(L.cell()[j]) : -1;
        if (c >= 0) mem[atomicSub(&ccs[c], 1) - 1] = (uint16_t)j;
    }
    __syncthreads();
    // members of each coarse cell by (column, id)
    for (int c = threadIdx.x; c < ncells; c += RES_THREADS) {
        const int a = ccs[c], b = ccs[c + 1];
        for (int m = a + 1; m < b; ++m) {
            const uint16_t v = mem[m];
            const uint32_t kx = L.cell()[v] & 0xffffu;
            const int ki = L.id()[v];
            int q = m - 1;
            while (q >= a) {
                const uint16_t u = mem[q];
                const uint32_t ux = L.cell()[u] & 0xffffu;
                if (ux < kx || (ux == kx && L.id()[u] < ki)) break;
                mem[q + 1] = u;
                --q;
            }
            mem[q + 1] = v;
        }
    }
    __syncthreads();
    const float h = R.hf, rv2 = R.rv2f;
    const float2 *off = L.off(X.cur);
    // pass 1 counts (per stencil row), pass 2 writes
    bool over = false;
    int e0 = 0;
    for (int pass = 0; pass < 2; ++pass) {
        for (int base = 0; base < X.p; base += RES_THREADS) {
            const int i = base + (int)threadIdx.x;
            int cnt = 0;
            if (i < X.p) {
                const uint32_t ci = L.cell()[i];
                const int cx = (int)(ci & 0xffffu), cy = (int)(ci >> 16);
                const float2 oi = off[i];
                uint32_t rows = 0;
                uint32_t e = pass ? L.lst()[i] : 0u;
                for (int oy = -1; oy <= 1; ++oy) {
                    const int ty = wrap1(cy + oy, nc);
                    const int grow = X.J.g == 1 ? ty : res_relrow(X, nc, cy) + oy;
                    const float sy = (float)oy * h - oi.y;
                    for (int ox = -1; ox <= 1 && grow >= 0 && grow < G; ++ox) {
                        const int tx = wrap1(cx + ox, nc);
                        const int cc = grow * ncol + tx / cw;
                        const float sx = (float)ox * h - oi.x;
                        const uint32_t tcell = (uint32_t)tx | ((uint32_t)ty << 16);
                        for (int m = ccs[cc]; m < ccs[cc + 1]; ++m) {
                            const int j = mem[m];
                            const uint32_t cj = L.cell()[j];
                            if ((cj & 0xffffu) > (uint32_t)tx) break;
                            if (cj != tcell || j == i) continue;
                            const float2 o = res_off(L, X.cur, pc, j);
                            const float rx = o.x + sx, ry = o.y + sy;
                            if (rx * rx + ry * ry < rv2) {
                                if (pass && (int)e < L.e_cap)
                                    L.ent()[e] = (uint16_t)((uint32_t)j | ((uint32_t)(ox + 1) << 14));
                                ++e;
                                ++cnt;
                            }
                        }
                    }
                    if (oy < 1) rows |= (uint32_t)min(cnt, 255) << (8 * (oy + 1));
                }
                if (!pass) {
                    L.rend()[i] = (uint16_t)rows;
                    over |= cnt > RES_MAXLIST;
                }
            }
            if (!pass) {
                int tot;
                const int at = e0 + block_excl_scan(cnt, s_w, &tot);
                if (i < X.p) L.lst()[i] = (uint32_t)at;
                e0 += tot;
            }
        }
        if (!pass) {
            if (threadIdx.x == 0) L.lst()[X.p] = (uint32_t)e0;
            over |= e0 > L.e_cap;
            if (__syncthreads_or(over)) {
                res_fail(&S.ctl->status, DS_CAPACITY);
                return false;
            }
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- rebuild
// Canonical cells for every own particle (the arithmetic of the global
// rebuild), then, with g > 1, the particles that left the slab's rows move
// to the neighbouring slab; the slab order of the rest is kept.
__device__ bool res_canon_migrate(const SysDev &S, const ResDev &D, const RepDev &R, const Slab &L,
                                  SlabRun &X, unsigned &my_gen, unsigned *bar, int *s_w) {
    const float h = R.hf;
    float2 *off = L.off(X.cur);
    for (int i = threadIdx.x; i < X.p; i += RES_THREADS) {
        float2 o = off[i];
        const uint32_t cpk = L.cell()[i];
        const int sx = o.x >= h ? 1 : (o.x < 0.0f ? -1 : 0);
        const int sy = o.y >= h ? 1 : (o.y < 0.0f ? -1 : 0);
        o.x -= (float)sx * h;
        o.y -= (float)sy * h;
        const int ncx = wrap1((int)(cpk & 0xffffu) + sx, R.nc);
        const int ncy = wrap1((int)(cpk >> 16) + sy, R.nc);
        off[i] = o;
        L.cell()[i] = (uint32_t)ncx | ((uint32_t)ncy << 16);
    }
    __syncthreads();
    if (X.J.g == 1) return true;
    // leaving through the top (row r1) -> direction 0, bottom (r0 - 1) -> 1;
    // stayers compacted in place, round by round (every read of a round
    // precedes its writes, and no write reaches a later round's slot)
    const int me = blockIdx.x;
    const int top = X.J.r1 == R.nc ? 0 : X.J.r1;
    int keep = 0, nout[2] = {0, 0};
    bool over = false;
    for (int base = 0; base < X.p; base += RES_THREADS) {
        const int i = base + (int)threadIdx.x;
        float2 o{}, v{};
        uint32_t c = 0;
        int id = 0, dir = -1;
        if (i < X.p) {
            o = off[i];
            v = L.vel()[i];
            c = L.cell()[i];
            id = L.id()[i];
            const int cy = (int)(c >> 16);
            if (!(cy >= X.J.r0 && cy < X.J.r1)) dir = cy == top ? 0 : 1;
        }
        int tk, t0, t1;
        const int ak = keep + block_excl_scan(i < X.p && dir < 0, s_w, &tk);
        const int a0 = nout[0] + block_excl_scan(dir == 0, s_w, &t0);
        const int a1 = nout[1] + block_excl_scan(dir == 1, s_w, &t1);
        if (i < X.p) {
            if (dir < 0) {
                off[ak] = o;
                L.vel()[ak] = v;
                L.cell()[ak] = c;
                L.id()[ak] = id;
            } else {
                const int at = dir == 0 ? a0 : a1;
                if (at < D.hmax) {
                    const long long gi = ((long long)me * 2 + dir) * D.hmax + at;
                    D.mig_a[gi] = make_float4(o.x, o.y, v.x, v.y);
                    D.mig_b[gi] = make_uint2(c, (uint32_t)id);
                } else {
                    over = true;
                }
            }
        }
        keep += tk;
        nout[0] += t0;
        nout[1] += t1;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        D.mig_n[me * 2] = nout[0];
        D.mig_n[me * 2 + 1] = nout[1];
    }
    if (__syncthreads_or(over)) res_fail(&S.ctl->status, DS_CAPACITY);
    if (!gang_sync(bar, X.J.g, my_gen, &S.ctl->status, S.timeout_ns)) return false;
    // arrivals: from the down neighbour's top (direction 0), then from the up
    // neighbour's bottom (direction 1)
    int p = keep;
    const int src[2] = {X.down, X.up};
    for (int q = 0; q < 2; ++q) {
        const int n = *(volatile int *)&D.mig_n[src[q] * 2 + q];
        if (p + n > X.J.p_cap) {
            res_fail(&S.ctl->status, DS_CAPACITY);
            return false;
        }
        for (int t = threadIdx.x; t < n; t += RES_THREADS) {
            const long long gi = ((long long)src[q] * 2 + q) * D.hmax + t;
            const float4 a = D.mig_a[gi];
            const uint2 b = D.mig_b[gi];
            off[p + t] = make_float2(a.x, a.y);
            L.vel()[p + t] = make_float2(a.z, a.w);
            L.cell()[p + t] = b.x;
            L.id()[p + t] = (int32_t)b.y;
        }
        p += n;
    }
    X.p = p;
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------- step
// Force on own particle i from its list (row by row, the column of each
// entry from its tag: the arithmetic of lj_list), then the velocity-Verlet
// update of kick_drift into the other own-offset buffer.
__device__ __forceinline__ void res_force_kick(const SysDev &S, const RepDev &R, const float *P, const Slab &L,
                                               const SlabRun &X, int i, bool first, bool dbg, float2 *pub0,
                                               float2 *pub1, float &vm, bool &bad) {
    const float2 *off = L.off(X.cur);
    const float2 *hoff = L.hoff();
    const uint16_t *ent = L.ent();
    const int pc = X.J.p_cap;
    const float2 oi = off[i];
    const float h = P[0], rc2 = P[1], eps24 = P[2], sig2 = P[3];
    const float sx0 = -h - oi.x, sx1 = -oi.x, sx2 = h - oi.x;
    const float sys[3] = {-h - oi.y, -oi.y, h - oi.y};
    const uint32_t st = L.lst()[i], en = L.lst()[i + 1];
    const uint32_t re = L.rend()[i];
    const uint32_t e1 = st + (re & 0xffu), e2 = st + (re >> 8);
    float fx = 0.0f, fy = 0.0f;
    double pe_unused = 0.0, fa_unused = 0.0;
    // batches of RES_U entries: all index and position loads of a batch are
    // issued before its pair arithmetic (latency hiding); the pairs are
    // still summed one by one in list order
    constexpr int RES_U = 4;
    for (uint32_t e = st; e < en; e += RES_U) {
        uint32_t v[RES_U];
        float2 o[RES_U];
#pragma unroll
        for (int u = 0; u < RES_U; ++u) v[u] = e + u < en ? (uint32_t)ent[e + u] : 0u;
#pragma unroll
        for (int u = 0; u < RES_U; ++u) {
            const int j = (int)(v[u] & RES_IDX);
            o[u] = j < pc ? off[j] : hoff[j - pc];
        }
#pragma unroll
        for (int u = 0; u < RES_U; ++u) {
            if (e + u < en) {
                const uint32_t t = v[u] >> 14;
                const float sx = t == 0 ? sx0 : (t == 1 ? sx1 : sx2);
                const float sy = e + u < e1 ? sys[0] : (e + u < e2 ? sys[1] : sys[2]);
                lj_pair_acc<float, false>(o[u].x + sx, o[u].y + sy, rc2, eps24, sig2, fx, fy, 0.0, pe_unused,
                                          fa_unused);
            }
        }
    }
    if (dbg) {
        S.dbg_fx[L.id()[i]] = (double)fx;
        S.dbg_fy[L.id()[i]] = (double)fy;
    }
    kick_drift<float>(R, oi, L.vel()[i], fx, fy, P[4], P[5], first, P[6], L.off(X.cur ^ 1), L.vel(), i, vm, bad);
    // a boundary particle's new offset goes straight to the neighbours' halo
    if (pub0) {
        const uint16_t b = L.bpos()[i];
        if (b != RES_NOB) (b >> 15 ? pub1 : pub0)[b & 0x7fffu] = L.off(X.cur ^ 1)[i];
    }
}

// Block maximum of v over the CTA into thread 0 (fixed order).
__device__ __forceinline__ float block_max(float v, float *s_f) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_f[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = 0.0f;
    if (threadIdx.x == 0)
        for (int w = 0; w < RES_THREADS / 32; ++w) m = fmaxf(m, s_f[w]);
    return m;
}

// ---------------------------------------------------------------- kernel
// Runs every slab job of this CTA for nsteps steps from step0.
__global__ void __launch_bounds__(RES_THREADS, RES_CTAS_PER_SM) k_md_resident(SysDev S, ResDev D, long long step0,
                                                                long long nsteps, int phase_half) {
    __shared__ int s_w[33];
    __shared__ float s_f[32];
    __shared__ double s_dm[2][32];
    __shared__ unsigned s_due;
    __shared__ long long s_win[MD_MAX_LG];
    __shared__ double s_disp;
    __shared__ int s_rebuild;
    __shared__ float s_par[8];   // the replica's FP32 constants: h, rc^2, 24 eps, sigma^2, dt/2m, dt, dt/(skin/2)
    Control *C = S.ctl;
    const int tid = threadIdx.x, lane = tid & 31;
    const int set = C->set, gcur = C->cur;
    const int per_lg = S.n_dx * S.nb;
    int *sh_hist = reinterpret_cast<int *>(res_smem);
    const uint32_t slab_base = (uint32_t)smem_hist_bytes(S.n_lg, S.n_dx, S.nb);
    const size_t avail = (size_t)D.smem_bytes - slab_base;
    for (int jb = D.job_start[blockIdx.x]; jb < D.job_start[blockIdx.x + 1]; ++jb) {
        SlabRun X;
        X.J = D.jobs[jb];
        const RepDev &R = S.reps[X.J.rep];
        const Slab L = res_layout(slab_base, X.J.p_cap, X.J.h_cap, avail);
        X.up = X.J.cta0 + (X.J.k + 1) % X.J.g;
        X.down = X.J.cta0 + (X.J.k + X.J.g - 1) % X.J.g;
        X.cur = 0;
        X.par = 0;
        unsigned *bar = D.gbar + 2 * (long long)X.J.rep;
        unsigned my_gen = 0;
        if (tid == 0) {
            my_gen = ld_acquire_gpu(&bar[1]);
            // the step's maximum starts from zero (a global-engine launch in
            // between leaves these slots untouched); before the first
            // barrier, so before any gang member adds to it
            if (X.J.k == 0) S.vmax_rep[(long long)X.J.rep * 3 + step0 % 3] = 0u;
            s_disp = S.disp_rep[X.J.rep];
            s_par[0] = R.hf;
            s_par[1] = R.rc2f;
            s_par[2] = 24.0f * R.epsf;   // the eps24 of lj_list
            s_par[3] = R.sig2f;
            s_par[4] = R.hkf;
            s_par[5] = R.dtf;
            s_par[6] = (float)(R.dt / R.half_skin);
        }
        for (int e = tid; e < S.n_lg * per_lg; e += RES_THREADS) sh_hist[e] = 0;
        if (!res_load(S, R, L, X, set, gcur, s_w)) {
            res_fail(&C->status, DS_CAPACITY);
            return;
        }
        if (!res_halo_full(S, D, R, L, X, my_gen, bar, s_w)) return;
        const uint64_t t_job = global_ns();   // the gang is together from here on
        if (!res_lists(S, R, L, X, s_w)) return;
        double m2acc[MD_MAX_LG], m4acc[MD_MAX_LG];
        for (long long it = 0; it < nsteps; ++it) {
            const long long s = step0 + it;
            if (tid == 0) {
                unsigned due = 0;
                const long long t = s + 1 - S.n_equil;
                for (int k = 0; k < S.n_lg; ++k) {
                    if (t >= 0 && t % S.lg_every[k] == 0) {
                        due |= 1u << k;
                        s_win[k] = t / S.lg_every[k] - 1;
                    } else {
                        s_win[k] = -1;
                    }
                }
                s_due = due;
                if (X.J.k == 0) S.vmax_rep[(long long)X.J.rep * 3 + (s + 1) % 3] = 0u;
            }
            const bool first = (it == 0) ? (phase_half == 0) : false;
            const bool dbg = S.dbg_fx && it == nsteps - 1;
            float vm = 0.0f;
            bool bad = false;
            const int nx = X.cur ^ 1, npar = X.par ^ 1;
            float2 *pub0 = nullptr, *pub1 = nullptr;
            if (X.J.g > 1) {
                pub0 = D.halo_off + (((long long)blockIdx.x * 2 + 0) * 2 + npar) * D.hmax;
                pub1 = D.halo_off + (((long long)blockIdx.x * 2 + 1) * 2 + npar) * D.hmax;
            }
            for (int i = tid; i < X.p; i += RES_THREADS)
                res_force_kick(S, R, s_par, L, X, i, first, dbg, pub0, pub1, vm, bad);
            if (__syncthreads_or(bad) && tid == 0) atomicOr(&C->status, (int)DS_NONFINITE);
            const float m = block_max(vm, s_f);
            if (tid == 0) atomicMax(&S.vmax_rep[(long long)X.J.rep * 3 + s % 3], __float_as_uint(m));
            if (!gang_sync(bar, X.J.g, my_gen, &C->status, S.timeout_ns)) return;
            if (tid == 0) {
                const unsigned v = *(volatile unsigned *)&S.vmax_rep[(long long)X.J.rep * 3 + s % 3];
                s_disp += (double)__uint_as_float(v) * 1.0000001;
                s_rebuild = s_disp >= 1.0;
            }
            if (X.J.g > 1) {
                const int src[2] = {X.up, X.down};
                for (int hh = 0; hh < 2; ++hh)
                    for (int t = tid; t < X.nh[hh]; t += RES_THREADS)
                        L.hoff()[hh * X.J.h_cap + t] =
                            D.halo_off[(((long long)src[hh] * 2 + hh) * 2 + npar) * D.hmax + t];
            }
            X.cur = nx;
            X.par = npar;
            __syncthreads();
            // ---- sampling pass (Eq. n_i), the arithmetic of the global engine
            const unsigned due = s_due;
            if (due) {
                for (int k = 0; k < S.n_lg; ++k) m2acc[k] = m4acc[k] = 0.0;
                for (int base = 0; base < X.p; base += RES_THREADS) {
                    const int i = base + tid;
                    const bool active = i < X.p;
                    int id = 0;
                    uint32_t cpk = 0;
                    float2 on{};
                    if (active) {
                        id = L.id()[i];
                        cpk = L.cell()[i];
                        on = L.off(X.cur)[i];
                    }
                    for (int k = 0; k < S.n_lg; ++k) {
                        if (!(due >> k & 1u)) continue;
                        const bool bin = s_win[k] >= 0;
                        int bins[MD_MAX_DX] = {-1, -1, -1, -1};
                        double m2 = 0.0, m4 = 0.0;
                        if (active) sample_particle<float>(S, R, X.J.rep, k, bin, id, cpk, on, bins, m2, m4);
                        if (bin) {
                            for (int d = 0; d < S.n_dx; ++d)
                                warp_hist_add(sh_hist + k * per_lg + d * S.nb, bins[d], lane);
                            m2acc[k] += m2;
                            m4acc[k] += m4;
                        }
                    }
                }
                for (int k = 0; k < S.n_lg; ++k) {
                    if (!(due >> k & 1u) || s_win[k] < 0) continue;
                    double a = m2acc[k], b = m4acc[k];
                    for (int o = 16; o > 0; o >>= 1) {
                        a += __shfl_xor_sync(0xffffffffu, a, o);
                        b += __shfl_xor_sync(0xffffffffu, b, o);
                    }
                    __syncthreads();
                    if (lane == 0) {
                        s_dm[0][tid >> 5] = a;
                        s_dm[1][tid >> 5] = b;
                    }
                    __syncthreads();
                    if (tid == 0) {
                        double ta = 0.0, tb = 0.0;
                        for (int w = 0; w < RES_THREADS / 32; ++w) {
                            ta += s_dm[0][w];
                            tb += s_dm[1][w];
                        }
                        double *mp = S.mom + ((long long)(R.pbase / 32 + X.J.k) * S.n_lg + k) * 2;
                        mp[0] += ta;
                        mp[1] += tb;
                    }
                }
                __syncthreads();
                flush_hist(S, sh_hist, X.J.rep, due, s_win);
                __syncthreads();
            }
            if (s_rebuild) {
                if (!res_canon_migrate(S, D, R, L, X, my_gen, bar, s_w)) return;
                if (!res_halo_full(S, D, R, L, X, my_gen, bar, s_w)) return;
                if (!res_lists(S, R, L, X, s_w)) return;
                if (tid == 0) {
                    s_disp = 0.0;
                    if (X.J.k == 0) atomicAdd((unsigned long long *)&C->n_rebuilds, 1ull);
                }
            }
            __syncthreads();
        }
        if (!res_store(S, D, R, L, X, set ^ 1, my_gen, bar)) return;
        if (tid == 0) D.job_ns[jb] = global_ns() - t_job;
        if (tid == 0 && X.J.k == 0) S.disp_rep[X.J.rep] = s_disp;
        __syncthreads();
    }
}

// After a resident launch: the state lives in the other set, unsorted (the
// global engine's cell lists are rebuilt before it is used again).  A
// separate launch, so that no CTA of the resident kernel can read the set
// index after it changed.
__global__ void k_res_flip(Control *C) {
    C->set ^= 1;
    C->cur = 0;
}

}  // namespace mdlg
