// Device side of the MD system: data layout, the persistent step kernel and
// the cell-list rebuild.  Included by md.cu only.
//
// Layout (all replicas of a batch back to back):
//   * slots: replica r owns slots [pbase_r, pbase_r + cap_r), cap_r = n_r
//     rounded up to SLOT_PAD; slots past n_r are padding, never active.
//   * particles are sorted by MD cell (row-major cy*nc + cx) within each
//     replica; cell_start[cbase_r + c] is the first slot of cell c.  Each
//     replica has one extra "padding cell" after its nc^2 cells that owns
//     its padding slots, so a single exclusive scan over all cells yields
//     every replica's cell_start.
//   * per slot: packed cell (cx | cy << 16), offset from the cell corner
//     (Vec2<T>, double-buffered: step s reads one buffer and writes the
//     other), velocity (Vec2<T>), particle id.  The four arrays come in two
//     sets; a rebuild gathers the sorted particles from one set into the
//     other.
//   * sampling snapshots are indexed by particle id: packed cell + offset.
#pragma once

#include "common.cuh"
#include "lattice.cuh"

namespace mdlg {

constexpr int SLOT_PAD = 256;   // slot padding per replica (multiple of every block size)
constexpr int GRAN = 128;       // slots per replica-lookup granule

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };

struct RepDev {
    int32_t nc, cbase, pbase, n, cap, ibase;
    int32_t lx[MD_MAX_DX];
    double h, L, dt, hk, rc2, eps, sig2, vshift, mass;
    double trig_lo, trig_hi;       // rebuild once an offset leaves [trig_lo, trig_hi)
    double dxl[MD_MAX_DX];
    float hf, dtf, hkf, rc2f, epsf, sig2f, trig_lof, trig_hif;
};

struct Control {
    unsigned bar_count, bar_gen;
    int status;
    int set, cur;
    int pad0;
    long long n_rebuilds;
    unsigned trig[3];
};

// Everything the kernels need, passed by value.
struct SysDev {
    const RepDev *reps;
    const int32_t *gran_rep;    // replica of each GRAN-slot granule
    Control *ctl;
    int32_t nslots, nrep, total_cells;
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
    // sampling
    uint32_t *snap_cell;        // [n_lg][ntot] by particle id
    void *snap_off;             // [n_lg][ntot] Vec2<T>
    int32_t *hist;              // [nrep][n_lg][n_dx][MD_NBLK][nb]
    unsigned long long *ovf;    // [nrep][n_lg][n_dx]
    double *mom;                // [nslots/32][n_lg][2]
    long long ntot;
    uint64_t timeout_ns;
};

template <typename T> __device__ __forceinline__ T rd(double d, float f);
template <> __device__ __forceinline__ double rd<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float rd<float>(double, float f) { return f; }

// Lennard-Jones force on the particle in slot `self` (packed cell cpk,
// offset oi) from all particles of the 3x3 block of cells around its cell
// (Sec. 4: V = 4 eps [(s/r)^12 - (s/r)^6] for r < rc; the force is the
// derivative of the unshifted potential).  The separation is
// (dcx*h + off_j - off_i) per axis: the stencil offset dcx carries the
// periodic image, so no wrap arithmetic is needed on positions.
template <typename T, bool kPE>
__device__ __forceinline__ void lj_stencil(const RepDev &R, const typename V2<T>::type *pos,
                                           const int32_t *cs, uint32_t cpk,
                                           typename V2<T>::type oi, int self, T &fx, T &fy,
                                           double &pe, double &fabs_sum) {
    const int nc = R.nc;
    const int cx = (int)(cpk & 0xffffu), cy = (int)(cpk >> 16);
    const T h = rd<T>(R.h, R.hf);
    const T rc2 = rd<T>(R.rc2, R.rc2f);
    const T eps = rd<T>(R.eps, R.epsf);
    const T sig2 = rd<T>(R.sig2, R.sig2f);
    const int32_t *csr = cs + R.cbase;
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
        const int row = wrap1(cy + oy, nc) * nc;
        const T sy = (T)oy * h - oi.y;
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
            const int c = row + wrap1(cx + ox, nc);
            const int s = csr[c], e = csr[c + 1];
            const T sx = (T)ox * h - oi.x;
            for (int j = s; j < e; ++j) {
                const typename V2<T>::type o = pos[j];
                const T rx = o.x + sx, ry = o.y + sy;
                const T r2 = rx * rx + ry * ry;
                if (r2 < rc2 && j != self) {
                    const T ir2 = T(1) / r2;
                    const T s2 = sig2 * ir2;
                    const T s6 = s2 * s2 * s2;
                    const T fr = T(24) * eps * s6 * (T(2) * s6 - T(1)) * ir2;
                    fx -= fr * rx;
                    fy -= fr * ry;
                    if (kPE) {
                        pe += 0.5 * (4.0 * (double)eps * ((double)s6 * (double)s6 - (double)s6) -
                                     R.vshift);
                        fabs_sum += fabs((double)fr) * sqrt((double)r2);
                    }
                }
            }
        }
    }
}

// ---------------------------------------------------------------- rebuild
// Counting sort of all particles by their current (canonical) MD cell, then
// particles inside one cell ordered by id, so the order -- and therefore
// every force sum -- is reproducible.  Six grid barriers.
template <typename T, int BLOCK>
__device__ bool rebuild(const SysDev &S, int &set, int &cur, unsigned &gen, int cbeg, int cend) {
    using V = typename V2<T>::type;
    Control *C = S.ctl;
    const int tid = threadIdx.x;
    const V *pos = static_cast<const V *>(S.pos[set][cur]);
    const uint32_t *cell = S.cell[set];
    // R1: new cell and rank inside it
    for (int ch = cbeg; ch < cend; ++ch) {
        const int slot = ch * BLOCK + tid;
        const RepDev &R = S.reps[S.gran_rep[slot / GRAN]];
        if (slot >= R.pbase + R.n) continue;
        const V o = pos[slot];
        const uint32_t cpk = cell[slot];
        const T h = rd<T>(R.h, R.hf);
        const int sx = o.x >= h ? 1 : (o.x < T(0) ? -1 : 0);
        const int sy = o.y >= h ? 1 : (o.y < T(0) ? -1 : 0);
        const int ncx = wrap1((int)(cpk & 0xffffu) + sx, R.nc);
        const int ncy = wrap1((int)(cpk >> 16) + sy, R.nc);
        const int gc = R.cbase + ncy * R.nc + ncx;
        S.newcell[slot] = gc;
        S.rank[slot] = atomicAdd(&S.cellcnt[gc], 1);
    }
    if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return false;
    // R2: per-CTA sums over a contiguous segment of cells
    const int seg = (S.total_cells + gridDim.x - 1) / gridDim.x;
    const int s0 = min(S.total_cells, (int)blockIdx.x * seg), s1 = min(S.total_cells, s0 + seg);
    {
        int acc = 0;
        for (int c = s0 + tid; c < s1; c += BLOCK) acc += S.cellcnt[c];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __shared__ int s_w[BLOCK / 32];
        if ((tid & 31) == 0) s_w[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < BLOCK / 32; ++w) t += s_w[w];
            S.blocksum[blockIdx.x] = t;
        }
    }
    if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return false;
    // R3: exclusive scan into cell_start
    {
        __shared__ int s_w[BLOCK / 32];
        __shared__ int s_base;
        int acc = 0;
        for (int b = tid; b < (int)blockIdx.x; b += BLOCK) acc += S.blocksum[b];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
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
    if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return false;
    // R4: scatter slot numbers to their new place; reset counts
    for (int ch = cbeg; ch < cend; ++ch) {
        const int slot = ch * BLOCK + tid;
        const RepDev &R = S.reps[S.gran_rep[slot / GRAN]];
        if (slot >= R.pbase + R.n)
            S.perm[slot] = -1;    // padding slots keep their place
        else
            S.perm[S.cell_start[S.newcell[slot]] + S.rank[slot]] = slot;
    }
    for (int c = s0 + tid; c < s1; c += BLOCK) S.cellcnt[c] = 0;
    if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return false;
    // R5: order each cell's particles by id; restore the padding-cell counts
    {
        const int32_t *pid = S.pid[set];
        for (int c = s0 + tid; c < s1; c += BLOCK) {
            const int a = S.cell_start[c], b = S.cell_start[c + 1];
            if (b - a < 2 || S.perm[a] < 0) continue;
            for (int i = a + 1; i < b; ++i) {
                const int pi = S.perm[i];
                const int key = pid[pi];
                int k = i - 1;
                while (k >= a && pid[S.perm[k]] > key) {
                    S.perm[k + 1] = S.perm[k];
                    --k;
                }
                S.perm[k + 1] = pi;
            }
        }
        for (int r = blockIdx.x * BLOCK + tid; r < S.nrep; r += gridDim.x * BLOCK) {
            const RepDev &R = S.reps[r];
            S.cellcnt[R.cbase + R.nc * R.nc] = R.cap - R.n;
        }
    }
    if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return false;
    // R6: gather into the other set with canonical offsets
    {
        const int ns = set ^ 1;
        V *npos = static_cast<V *>(S.pos[ns][0]);
        V *nvel = static_cast<V *>(S.vel[ns]);
        const V *vel = static_cast<const V *>(S.vel[set]);
        const int32_t *pid = S.pid[set];
        for (int ch = cbeg; ch < cend; ++ch) {
            const int slot = ch * BLOCK + tid;
            const RepDev &R = S.reps[S.gran_rep[slot / GRAN]];
            if (slot >= R.pbase + R.n) continue;
            const int old = S.perm[slot];
            V o = pos[old];
            const uint32_t cpk = cell[old];
            const T h = rd<T>(R.h, R.hf);
            const int sx = o.x >= h ? 1 : (o.x < T(0) ? -1 : 0);
            const int sy = o.y >= h ? 1 : (o.y < T(0) ? -1 : 0);
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
    if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return false;
    set ^= 1;
    cur = 0;
    if (blockIdx.x == 0 && tid == 0) C->n_rebuilds += 1;
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

// ---------------------------------------------------------------- persistent step kernel
// Advances all replicas by nsteps velocity-Verlet steps.  Per step and slot:
// force F_s at the current offsets; v += (dt/2m) F twice (the first kick
// completes the previous step unless velocities are at an integer step);
// off += dt v into the other position buffer; on sampling steps the new
// position is binned against the particle's snapshot (Eq. n_i) and becomes
// the new snapshot.  One grid barrier per step; a cell-list rebuild follows
// any step after which a particle strayed 0.45 skin outside its cell.
template <typename T, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_md_persistent(SysDev S, long long step0, long long nsteps,
                                                         int phase_half, int force_rebuild) {
    using V = typename V2<T>::type;
    extern __shared__ int sh_hist[];
    __shared__ unsigned s_due;
    __shared__ long long s_win[MD_MAX_LG];
    __shared__ int s_trig;
    Control *C = S.ctl;
    const int tid = threadIdx.x, lane = tid & 31;
    unsigned gen = 0;
    if (tid == 0) gen = ld_acquire_gpu(&C->bar_gen);
    int set = C->set, cur = C->cur;
    const int nchunks = S.nslots / BLOCK;
    const int q = (nchunks + gridDim.x - 1) / gridDim.x;
    const int cbeg = min(nchunks, (int)blockIdx.x * q), cend = min(nchunks, cbeg + q);
    const int per_lg = S.n_dx * S.nb;
    for (int e = tid; e < S.n_lg * per_lg; e += BLOCK) sh_hist[e] = 0;

    if (force_rebuild) {
        if (!rebuild<T, BLOCK>(S, set, cur, gen, cbeg, cend)) return;
    }
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
            s_trig = 0;
            if (blockIdx.x == 0) C->trig[(s + 1) % 3] = 0u;
        }
        __syncthreads();
        const unsigned due = s_due;
        const bool first = (it == 0) ? (phase_half == 0) : false;
        const V *pin = static_cast<const V *>(S.pos[set][cur]);
        V *pout = static_cast<V *>(S.pos[set][cur ^ 1]);
        V *vel = static_cast<V *>(S.vel[set]);
        const uint32_t *cell = S.cell[set];
        const int32_t *pid = S.pid[set];
        int hist_rep = -1;
        bool trig = false;
        for (int ch = cbeg; ch < cend; ++ch) {
            const int slot = ch * BLOCK + tid;
            const int rep = S.gran_rep[(ch * BLOCK) / GRAN];
            const RepDev &R = S.reps[rep];
            if (due && rep != hist_rep) {
                if (hist_rep >= 0) {
                    __syncthreads();
                    flush_hist(S, sh_hist, hist_rep, due, s_win);
                    __syncthreads();
                }
                hist_rep = rep;
            }
            const bool active = slot < R.pbase + R.n;
            V on;
            uint32_t cpk = 0;
            int myid = 0;
            if (active) {
                const V oi = pin[slot];
                cpk = cell[slot];
                V v = vel[slot];
                T fx = T(0), fy = T(0);
                double pe_unused = 0.0, fa_unused = 0.0;
                lj_stencil<T, false>(R, pin, S.cell_start, cpk, oi, slot, fx, fy, pe_unused,
                                     fa_unused);
                const T hk = rd<T>(R.hk, R.hkf), dt = rd<T>(R.dt, R.dtf);
                if (!first) {
                    v.x = v.x + hk * fx;
                    v.y = v.y + hk * fy;
                }
                v.x = v.x + hk * fx;
                v.y = v.y + hk * fy;
                on.x = oi.x + dt * v.x;
                on.y = oi.y + dt * v.y;
                pout[slot] = on;
                vel[slot] = v;
                const T lo = rd<T>(R.trig_lo, R.trig_lof), hi = rd<T>(R.trig_hi, R.trig_hif);
                if (!(on.x >= lo && on.x < hi && on.y >= lo && on.y < hi)) {
                    trig = true;
                    const T h = rd<T>(R.h, R.hf);
                    // not finite, or more than one cell beyond its own cell
                    if (!(on.x >= -h && on.x < T(2) * h && on.y >= -h && on.y < T(2) * h))
                        atomicOr(&C->status, isfinite((double)on.x) && isfinite((double)on.y)
                                                 ? (int)DS_SKIN
                                                 : (int)DS_NONFINITE);
                }
                if (due) myid = pid[slot];
            }
            if (due) {
                // MDLG sampling of this step's new positions
                for (int k = 0; k < S.n_lg; ++k) {
                    if (!(due >> k & 1u)) continue;
                    double m2 = 0.0, m4 = 0.0;
                    uint32_t *scell = S.snap_cell + (long long)k * S.ntot;
                    V *soff = static_cast<V *>(S.snap_off) + (long long)k * S.ntot;
                    int bins[MD_MAX_DX];
#pragma unroll
                    for (int d = 0; d < MD_MAX_DX; ++d) bins[d] = -1;
                    if (active) {
                        const int cx = (int)(cpk & 0xffffu), cy = (int)(cpk >> 16);
                        if (s_win[k] >= 0) {
                            const uint32_t spk = scell[myid];
                            const V so = soff[myid];
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
                            const double x1 = cell_position(cx, R.h, (double)on.x);
                            const double y1 = cell_position(cy, R.h, (double)on.y);
                            const double x0 = cell_position(scx, R.h, (double)so.x);
                            const double y0 = cell_position(scy, R.h, (double)so.y);
                            for (int d = 0; d < S.n_dx; ++d) {
                                const int lx = R.lx[d];
                                const double dxl = R.dxl[d];
                                const long long ddx =
                                    lattice_shift(lattice_cell(x1, dxl, lx) - lattice_cell(x0, dxl, lx), lx);
                                const long long ddy =
                                    lattice_shift(lattice_cell(y1, dxl, lx) - lattice_cell(y0, dxl, lx), lx);
                                if (ddx >= -S.W && ddx <= S.W && ddy >= -S.W && ddy <= S.W)
                                    bins[d] = (int)((ddy + S.W) * (2 * S.W + 1) + (ddx + S.W));
                                else
                                    atomicAdd(&S.ovf[((long long)rep * S.n_lg + k) * S.n_dx + d], 1ull);
                            }
                        }
                        scell[myid] = cpk;
                        soff[myid] = on;
                    }
                    if (s_win[k] >= 0) {
                        for (int d = 0; d < S.n_dx; ++d)
                            warp_hist_add(sh_hist + k * per_lg + d * S.nb, bins[d], lane);
                        for (int o = 16; o > 0; o >>= 1) {
                            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
                            m4 += __shfl_xor_sync(0xffffffffu, m4, o);
                        }
                        if (lane == 0) {
                            double *mp = S.mom + ((long long)(slot >> 5) * S.n_lg + k) * 2;
                            mp[0] += m2;
                            mp[1] += m4;
                        }
                    }
                }
            }
        }
        if (due && hist_rep >= 0) {
            __syncthreads();
            flush_hist(S, sh_hist, hist_rep, due, s_win);
        }
        if (__syncthreads_or(trig) && tid == 0) atomicOr(&C->trig[s % 3], 1u);
        if (!grid_sync({&C->bar_count, &C->bar_gen, &C->status}, gen, S.timeout_ns)) return;
        cur ^= 1;
        if (*(volatile unsigned *)&C->trig[s % 3]) {
            if (!rebuild<T, BLOCK>(S, set, cur, gen, cbeg, cend)) return;
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        C->set = set;
        C->cur = cur;
    }
}

// ---------------------------------------------------------------- observation kernel
// One pass at the current step without moving particles: forces, optional
// completion of the half kick (velocities then refer to the current step),
// per-warp energy/momentum partials, and outputs in particle-id order.
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
            lj_stencil<T, true>(R, pos, S.cell_start, cpk, oi, slot, fx, fy, pe, fa);
            if (A.complete) {
                const T hk = rd<T>(R.hk, R.hkf);
                v.x = v.x + hk * fx;
                v.y = v.y + hk * fy;
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
