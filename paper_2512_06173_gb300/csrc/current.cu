// K1b: molecular current density J^{n+1/2} = sum_m gamma_m mudot_m kappa_m on a
// dense box (Eq. J_mol with Eq. Polarization_mol).
//
// The box is the bounding box of all molecules' kernel windows; it is tiled into
// blocks of JX x JY x JZ cells.  Each block owns a list of (molecule, window start
// relative to the block) entries, built once when molecules are added.  Because
// the Gaussian kernel is separable,
//     J_c(x, y, k) = sum_e  Bx_e(x) * G_e(y, k),   G_e(y, k) = gamma mudot_e^c Ay_e(y) Cz_e(k),
// with the 1D weights at the staggering of component c.  Per batch of entries the
// block stages Bx (dense over the 32 columns, zero outside the window) and G (dense
// over JY x JZ) in shared memory; each thread then accumulates the JZ cells of its
// (x, y) column with one FMA per entry and cell.  The sum runs in the fixed order
// of the block's list: deterministic, no atomics.  Only components along which
// some molecule has a dipole are computed (cmask).
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

template <typename T>
__device__ __forceinline__ T rec_value(const int4 en, const int wfm, const T *w, const int c, const int q) {
    int axis, d;
    if (q < JX) { axis = 0; d = q - en.y; }
    else if (q < JX + JY) { axis = 1; d = q - JX - en.z; }
    else { axis = 2; d = q - JX - JY - en.w; }
    const int W = (wfm >> (8 * axis)) & 0xff;
    return ((unsigned)d < (unsigned)W) ? w[(long long)en.x * NW + (2 * axis + (axis == c ? 1 : 0)) * WMAX + d] : T(0);
}

template <typename T>
__device__ __forceinline__ void current_body(const CurArgs<T> &a, const int blk) {
    constexpr int JEB = sizeof(T) == 4 ? 32 : 16;  // entries staged per batch
    __shared__ __align__(16) T sR[JEB][RC];
    __shared__ __align__(16) T sG[JEB][JY][JZ];
    __shared__ T sC[JEB];
    __shared__ int4 sEnt[JEB];
    __shared__ int sWf[JEB];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * JX + tx;
    const int beg = a.off[blk], end = a.off[blk + 1];
    if (beg == end) return;  // no window here: J stays 0 (the box is zeroed at setup)
    const int bx = blk % a.nbx, by = (blk / a.nbx) % a.nby, bz = blk / (a.nbx * a.nby);
    const int xr = bx * JX + tx, yr = by * JY + ty, zr0 = bz * JZ;
    for (int c = 0; c < 3; c++) {
        if (!((a.cmask >> c) & 1)) continue;
        T acc[JZ];
#pragma unroll
        for (int q = 0; q < JZ; q++) acc[q] = T(0);
        for (int base = beg; base < end; base += JEB) {
            const int nb = min(JEB, end - base);
            __syncthreads();  // previous batch fully consumed
            if (tid < nb) {
                const int4 en = a.ent[base + tid];
                sEnt[tid] = en;
                sWf[tid] = a.wf[en.x];
                sC[tid] = a.c[3ll * en.x + c];
            }
            __syncthreads();
            for (int t = tid; t < nb * RC; t += JX * JY) sR[t / RC][t % RC] = rec_value(sEnt[t / RC], sWf[t / RC], a.w, c, t % RC);
            __syncthreads();
            // G_e(y, k) = gamma mudot_e^c Ay_e(y) Cz_e(k)
            for (int t = tid; t < nb * JY * JZ; t += JX * JY) {
                const int e = t / (JY * JZ), r = t % (JY * JZ), yy = r / JZ, zz = r % JZ;
                sG[e][yy][zz] = sC[e] * sR[e][JX + yy] * sR[e][JX + JY + zz];
            }
            __syncthreads();
            for (int e = 0; e < nb; e++) {
                const T b = sR[e][tx];
#pragma unroll
                for (int q = 0; q < JZ; q++) acc[q] += b * sG[e][ty][q];
            }
        }
        if (xr < a.bn[0] && yr < a.bn[1]) {
            T *out = a.J[c];
#pragma unroll
            for (int q = 0; q < JZ; q++) {
                const int zr = zr0 + q;
                if (zr < a.bn[2]) out[((long long)zr * a.bn[1] + yr) * a.bn[0] + xr] = acc[q];
            }
        }
    }
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
__global__ void __launch_bounds__(JX *JY) current_kernel(const CurArgs<T> a) {
    pdl_trigger();
    pdl_wait();
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
__global__ void __launch_bounds__(JX *JY) current_batch_kernel(const CurBatch<T> b) {
    pdl_trigger();
    pdl_wait();
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
