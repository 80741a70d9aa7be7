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

namespace ml {


template <typename T>
__global__ void __launch_bounds__(JX *JY) current_kernel(const CurArgs<T> a) {
    constexpr int JEB = sizeof(T) == 4 ? 64 : 32;  // entries staged per batch
    __shared__ T sB[JEB][JX];
    __shared__ __align__(16) T sG[JEB][JY][JZ];
    __shared__ int4 sE[JEB];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * JX + tx;
    const int blk = blockIdx.x;
    const int bx = blk % a.nbx, by = (blk / a.nbx) % a.nby, bz = blk / (a.nbx * a.nby);
    const int beg = a.off[blk], end = a.off[blk + 1];
    // box-relative cell of this thread's column
    const int xr = bx * JX + tx, yr = by * JY + ty, zr0 = bz * JZ;
    for (int c = 0; c < 3; c++) {
        if (!((a.cmask >> c) & 1)) continue;
        // staggering of component c: half-integer along c, integer elsewhere
        const int sxo = (c == 0 ? WMAX : 0), syo = 2 * WMAX + (c == 1 ? WMAX : 0), szo = 4 * WMAX + (c == 2 ? WMAX : 0);
        T acc[JZ];
#pragma unroll
        for (int q = 0; q < JZ; q++) acc[q] = T(0);
        for (int base = beg; base < end; base += JEB) {
            const int nb = min(JEB, end - base);
            __syncthreads();  // previous batch fully consumed
            if (tid < nb) sE[tid] = a.ent[base + tid];
            __syncthreads();
            // Bx: entry e per thread row group, column tx
            for (int e = ty; e < nb; e += JY) {
                const int4 en = sE[e];
                const int wf = a.wf[en.x];
                const int dx = tx - en.y;
                sB[e][tx] = ((unsigned)dx < (unsigned)(wf & 0xff)) ? a.w[(long long)en.x * NW + sxo + dx] : T(0);
            }
            // G: entries x (JY x JZ) values
            for (int t = tid; t < nb * JY * JZ; t += JX * JY) {
                const int e = t / (JY * JZ), r = t % (JY * JZ), yy = r / JZ, zz = r % JZ;
                const int4 en = sE[e];
                const int wf = a.wf[en.x];
                const int dy = yy - en.z, dz = zz - en.w;
                T g = T(0);
                if ((unsigned)dy < (unsigned)((wf >> 8) & 0xff) && (unsigned)dz < (unsigned)((wf >> 16) & 0xff)) {
                    const T *w = a.w + (long long)en.x * NW;
                    g = a.c[3ll * en.x + c] * w[syo + dy] * w[szo + dz];
                }
                sG[e][yy][zz] = g;
            }
            __syncthreads();
            for (int e = 0; e < nb; e++) {
                const T b = sB[e][tx];
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

template <typename T>
cudaError_t launch_current(const CurArgs<T> &a, cudaStream_t s) {
    if (a.nblocks == 0) return cudaSuccess;
    current_kernel<T><<<a.nblocks, dim3(JX, JY), 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_current<float>(const CurArgs<float> &, cudaStream_t);
template cudaError_t launch_current<double>(const CurArgs<double> &, cudaStream_t);

}  // namespace ml
