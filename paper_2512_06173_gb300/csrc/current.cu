// K1b: molecular current density J^{n+1/2} = sum_m gamma_m mudot_m kappa_m on a
// dense box (Eq. J_mol with Eq. Polarization_mol).
//
// The box is the bounding box of all molecules' kernel windows; it is tiled into
// blocks of JX x JY x JZ cells.  Each block owns a list of (molecule, window start
// relative to the block) entries, built once when molecules are added.  Because
// the Gaussian kernel is separable,
//     J_c(x, y, k) = sum_e  Bx_e(x) * G_e(y, k),   G_e(y, k) = gamma mudot_e^c Ay_e(y) Cz_e(k),
// with the 1D weights at the staggering of component c.  Per batch of entries the
// block stages the entries' 1D records (Bx dense over the 32 columns, gamma mudot Ay
// over JY rows, Cz over JZ planes, zero outside the window) in shared memory; each
// thread accumulates its 4 x 2 cells with one FMA per entry and cell, and a warp skips
// the entries whose x window misses its columns.  The sum runs in the fixed order of
// the block's list: deterministic, no atomics.  Only components along which some
// molecule has a dipole are computed (cmask).
#include "ml_internal.cuh"
#include "tma.cuh"

namespace ml {


// Weight record of entry en (molecule en.x, window start relative to the block
// origin en.y, en.z, en.w) for component c, slot q of RC = JX + JY + JZ:
//   [0, JX) Bx(x)   [JX, JX+JY) Ay(y)   [JX+JY, RC) Cz(z),
// each the molecule's 1D weight at the block's own cell (half-integer position along
// c, integer elsewhere), 0 outside the window.  Built in shared memory per batch of
// entries from the per-molecule weight table, which stays in L2.
constexpr int RC = JX + JY + JZ;
static_assert(JX == 32 && JY == 8 && JZ == 8, "current_body maps 8 warps x 32 lanes onto 32 x 8 x 8 cells");

template <typename T>
__device__ __forceinline__ T rec_value(const int4 en, const int wfm, const T *w, const int c, const int q) {
    int axis, d;
    if (q < JX) { axis = 0; d = q - en.y; }
    else if (q < JX + JY) { axis = 1; d = q - JX - en.z; }
    else { axis = 2; d = q - JX - JY - en.w; }
    const int W = (wfm >> (8 * axis)) & 0xff;
    return ((unsigned)d < (unsigned)W) ? w[(long long)en.x * NW + (2 * axis + (axis == c ? 1 : 0)) * WMAX + d] : T(0);
}

// Thread layout: warp w owns the four columns x = 4w .. 4w+3 of the block; lane l the
// row y = l & 7 and the planes z = (l >> 3) and (l >> 3) + 4, so a thread holds 4 x 2
// cells.  When a batch of entries is staged, one ballot per warp over the entries'
// column masks (built with the lists) marks the entries whose x window meets that
// warp's columns; a warp then visits only its marked entries, in list order (an
// unmarked entry has Bx = 0 there).  The per-cell sum is that of the dense form, entry
// by entry in list order: acc += Bx * ((c Ay) Cz).
// Records are built one entry per warp (lane q: Bx at column q; lanes 0..15: Ay and Cz)
// with every load of the batch issued before the first store, straight from the
// weight table (zero past each window, so the bound is WMAX).  Nothing before the
// amplitudes depends on the molecule kernel: when launched as its programmatic
// dependent, a block stages its entries and records first and waits only before it
// reads c.  The block's cells leave through a padded shared tile so that the global
// stores are whole rows.
template <typename T>
__device__ __forceinline__ void current_body(const CurArgs<T> &a, const int blk) {
    constexpr int JEB = sizeof(T) == 4 ? 128 : 64;  // entries staged per batch (128: 0.153 vs 0.158 ms at 96 on the 512 x 512 x 384 ensemble)
    constexpr int NWD = JEB / 32;                   // ballot words per warp
    constexpr int KE = JEB / JY;                    // entries whose records one warp builds
    constexpr int TXP = JX + 4;                     // padded row of the output tile
    __shared__ __align__(16) T sR[JEB][RC];         // Bx | Ay | Cz per entry
    __shared__ __align__(16) T sT[JZ][JY][TXP];
    __shared__ int4 sEnt[JEB];
    __shared__ T sC[JEB];
    __shared__ unsigned sMask[JX / 4][NWD];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * JX + tx;
    const int beg = a.off[blk], end = a.off[blk + 1];
    if (beg == end) {  // no window here: J stays 0 (the box is zeroed at setup)
        pdl_wait();
        return;
    }
    const int bx = blk % a.nbx, by = (blk / a.nbx) % a.nby, bz = blk / (a.nbx * a.nby);
    const int w = ty, ly = tx & 7, lz = tx >> 3;
    bool waited = false;
    for (int c = 0; c < 3; c++) {
        if (!((a.cmask >> c) & 1)) continue;
        const int ox = (c == 0 ? 1 : 0) * WMAX, oy = (2 + (c == 1 ? 1 : 0)) * WMAX, oz = (4 + (c == 2 ? 1 : 0)) * WMAX;
        T acc[4][2];
#pragma unroll
        for (int k = 0; k < 4; k++) acc[k][0] = acc[k][1] = T(0);
        for (int base = beg; base < end; base += JEB) {
            const int nb = min(JEB, end - base);
            __syncthreads();  // previous batch (and the previous component's tile) consumed
            if (ty < NWD) {
                const bool has = tid < nb;
                unsigned mk = 0;
                if (has) {
                    sEnt[tid] = a.ent[base + tid];
                    mk = a.emask[base + tid];
                }
#pragma unroll
                for (int q = 0; q < JX / 4; q++) {
                    const unsigned bal = __ballot_sync(0xffffffffu, (mk >> q) & 1u);
                    if (tx == 0) sMask[q][ty] = bal;
                }
            }
            __syncthreads();
            T vx[KE], vyz[KE];
#pragma unroll
            for (int k = 0; k < KE; k++) {
                const int e = ty + JY * k;
                vx[k] = vyz[k] = T(0);
                if (e < nb) {
                    const int4 en = sEnt[e];
                    const T *wm = a.w + (long long)en.x * NW;
                    int d = tx - en.y;
                    if ((unsigned)d < (unsigned)WMAX) vx[k] = wm[ox + d];
                    if (tx < JY) {
                        d = tx - en.z;
                        if ((unsigned)d < (unsigned)WMAX) vyz[k] = wm[oy + d];
                    } else if (tx < JY + JZ) {
                        d = tx - JY - en.w;
                        if ((unsigned)d < (unsigned)WMAX) vyz[k] = wm[oz + d];
                    }
                }
            }
            if (!waited) {
                pdl_wait();  // the amplitudes of this step are complete
                waited = true;
            }
            const T cv = tid < nb ? a.c[3ll * sEnt[tid].x + c] : T(0);
#pragma unroll
            for (int k = 0; k < KE; k++) {
                const int e = ty + JY * k;
                if (e < nb) {
                    sR[e][tx] = vx[k];
                    if (tx < JY + JZ) sR[e][JX + tx] = vyz[k];
                }
            }
            if (tid < nb) sC[tid] = cv;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NWD; q++) {
                unsigned bits = sMask[w][q];
                while (bits) {
                    const int e = 32 * q + __ffs(bits) - 1;
                    bits &= bits - 1;
                    T b[4];
                    if constexpr (sizeof(T) == 4) {
                        const float4 v = *reinterpret_cast<const float4 *>(&sR[e][4 * w]);
                        b[0] = v.x; b[1] = v.y; b[2] = v.z; b[3] = v.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; k++) b[k] = sR[e][4 * w + k];
                    }
                    const T cay = sC[e] * sR[e][JX + ly];
                    const T p0 = cay * sR[e][JX + JY + lz], p1 = cay * sR[e][JX + JY + lz + 4];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        acc[k][0] += b[k] * p0;
                        acc[k][1] += b[k] * p1;
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            sT[lz][ly][4 * w + k] = acc[k][0];
            sT[lz + 4][ly][4 * w + k] = acc[k][1];
        }
        __syncthreads();
        const int xr = bx * JX + tx, yr = by * JY + ty;
        if (xr < a.bn[0] && yr < a.bn[1]) {
            T *out = c == 0 ? a.J[0] : (c == 1 ? a.J[1] : a.J[2]);  // no dynamic index into the parameter
#pragma unroll
            for (int q = 0; q < JZ; q++) {
                const int zr = bz * JZ + q;
                if (zr < a.bn[2]) out[((long long)zr * a.bn[1] + yr) * a.bn[0] + xr] = sT[q][ty][tx];
            }
        }
    }
    if (!waited) pdl_wait();
}

// Gather (Eq. E_regu_Emi), the transpose of the current kernel over the same
// blocks, entry lists and records: the block stages E^n of its JX x JY x JZ cells
// (coalesced), then one warp per entry forms, lane x,
//     T(x) = sum_k Cz_e(k) sum_y Ay_e(y) E(x, y, k)
// and reduces sum_x Bx_e(x) T(x) with a fixed xor-shuffle tree.  The partial of
// entry e and component c goes to part[e][c]; nothing is accumulated across
// blocks here, so the result does not depend on scheduling.
template <typename T>
__device__ __forceinline__ void gather_body(const GathArgs<T> &a, const int blk) {
    constexpr int JEB = sizeof(T) == 4 ? 32 : 16;
    __shared__ __align__(16) T sE[JZ][JY][JX];
    __shared__ __align__(16) T sR[JEB][RC];
    __shared__ int4 sEnt[JEB];
    __shared__ int sWf[JEB];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * JX + tx;
    const int beg = a.off[blk], end = a.off[blk + 1];
    if (beg == end) return;
    const int bx = blk % a.nbx, by = (blk / a.nbx) % a.nby, bz = blk / (a.nbx * a.nby);
    const int xr = bx * JX + tx, yr0 = by * JY, zr0 = bz * JZ;
    for (int c = 0; c < 3; c++) {
        if (!((a.gcmask >> c) & 1)) continue;
        __syncthreads();  // sE of the previous component consumed
        for (int q = ty; q < JY * JZ; q += JY) {
            const int yy = q % JY, zz = q / JY;
            const int yr = yr0 + yy, zr = zr0 + zz;
            T v = T(0);
            if (xr < a.bn[0] && yr < a.bn[1] && zr < a.bn[2]) {
                const long long g = (long long)(a.b0[2] + zr + 1) * a.plane + (long long)(a.b0[1] + yr + 1) * a.px +
                                    (a.b0[0] + xr + XO);
                v = a.E[c][g];
            }
            sE[zz][yy][tx] = v;
        }
        for (int base = beg; base < end; base += JEB) {
            const int nb = min(JEB, end - base);
            __syncthreads();  // previous batch consumed (and sE written)
            if (tid < nb) {
                const int4 en = a.ent[base + tid];
                sEnt[tid] = en;
                sWf[tid] = a.wf[en.x];
            }
            __syncthreads();
            for (int t = tid; t < nb * RC; t += JX * JY) sR[t / RC][t % RC] = rec_value(sEnt[t / RC], sWf[t / RC], a.w, c, t % RC);
            __syncthreads();
            for (int e = ty; e < nb; e += JY) {
                const int m = sEnt[e].x;
                T v = T(0);
                if ((a.cmask[m] >> c) & 1) {
                    T t = T(0);
#pragma unroll
                    for (int zz = 0; zz < JZ; zz++) {
                        T u = T(0);
#pragma unroll
                        for (int yy = 0; yy < JY; yy++) u += sR[e][JX + yy] * sE[zz][yy][tx];
                        t += sR[e][JX + JY + zz] * u;
                    }
                    v = sR[e][tx] * t;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (tx == 0) a.part[3ll * (base + e) + c] = v;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(JX *JY) gather_kernel(const GathArgs<T> a) { gather_body(a, (int)blockIdx.x); }

// The field pass may be launched as this kernel's programmatic dependent: release it at
// once (only its current-box tiles wait for this kernel's completion).  When this kernel
// is itself launched that way, wait for the molecule kernel before reading its output.
template <typename T>
__global__ void __launch_bounds__(JX *JY, 4) current_kernel(const CurArgs<T> a) {
    pdl_trigger();
    current_body(a, (int)blockIdx.x);
}

// Batched forms: one block per (instance, box block) work item; the gather reads the
// time level of this step.
template <typename T>
__global__ void __launch_bounds__(JX *JY) gather_batch_kernel(const GathBatch<T> b) {
    const int2 wk = b.work[blockIdx.x];
    gather_body(b.args[2 * wk.x + ((b.lev0[wk.x] + b.s) & 1)], wk.y);
}

template <typename T>
__global__ void __launch_bounds__(JX *JY, 4) current_batch_kernel(const CurBatch<T> b) {
    pdl_trigger();
    const int2 wk = b.work[blockIdx.x];
    current_body(b.args[wk.x], wk.y);
}

template <typename T>
cudaError_t launch_gather_batch(const GathBatch<T> &b, int nwork, cudaStream_t s) {
    if (nwork == 0) return cudaSuccess;
    gather_batch_kernel<T><<<nwork, dim3(JX, JY), 0, s>>>(b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_current_batch(const CurBatch<T> &b, int nwork, cudaStream_t s, bool pdl) {
    if (nwork == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nwork);
    cfg.blockDim = dim3(JX, JY);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, current_batch_kernel<T>, b);
}

template <typename T>
cudaError_t launch_gather(const GathArgs<T> &a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    gather_kernel<T><<<a.nblocks, dim3(JX, JY), 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_current(const CurArgs<T> &a, cudaStream_t s, bool pdl) {
    if (a.nblocks == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.nblocks);
    cfg.blockDim = dim3(JX, JY);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, current_kernel<T>, a);
}

#define ML_INST(T)                                                                                 \
    template cudaError_t launch_current<T>(const CurArgs<T> &, cudaStream_t, bool);                \
    template cudaError_t launch_gather<T>(const GathArgs<T> &, cudaStream_t);                      \
    template cudaError_t launch_gather_batch<T>(const GathBatch<T> &, int, cudaStream_t);          \
    template cudaError_t launch_current_batch<T>(const CurBatch<T> &, int, cudaStream_t, bool);    \

ML_INST(float)
ML_INST(double)

}  // namespace ml
