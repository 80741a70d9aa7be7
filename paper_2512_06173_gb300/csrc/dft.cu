// K4: DFT flux planes.  The transmitted-flux spectra of Sec. IV.C/IV.D are
// Re sum_plane (E~ x H~*) . n with E~(w) = sum_n E^{n+1} e^{i w (n+1) dt} dt and
// H~(w) = sum_n H^{n+1/2} e^{i w (n+1/2) dt} dt.  Instead of touching FP64
// accumulators of every frequency each step (a read-modify-write of 16 B x 4
// components x nfreq per plane cell per step), each step only copies the four
// tangential plane components into a K-deep FP32/FP64 sample ring; every K steps
// the fold kernel adds the K samples, with phases computed in FP64 from the
// absolute step index, into FP64 accumulators.  Same sums, regrouped.
#include "ml_internal.cuh"

namespace ml {

constexpr int DFT_K = DFT_KMAX;

template <typename T>
__global__ void dft_sample_kernel(const PlaneArgs<T> a) {
    const int ncell = a.nb * a.nc;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    const int u = t % a.nb, v = t / a.nb;
    const int b = (a.axis + 1) % 3, c = (a.axis + 2) % 3;
    int idx[3], idm[3];
    idx[a.axis] = a.index; idx[b] = u; idx[c] = v;
    idm[a.axis] = a.index - 1; idm[b] = u; idm[c] = v;
    const long long g = (long long)(idx[2] + 1) * a.plane + (long long)(idx[1] + 1) * a.px + (idx[0] + XO);
    const long long gm = (long long)(idm[2] + 1) * a.plane + (long long)(idm[1] + 1) * a.px + (idm[0] + XO);
    T *out = a.buf + (long long)a.slot * 4 * ncell;
    out[t] = a.E[b][g];
    out[ncell + t] = a.E[c][g];
    out[2 * ncell + t] = T(0.5) * (a.H[b][g] + a.H[b][gm]);
    out[3 * ncell + t] = T(0.5) * (a.H[c][g] + a.H[c][gm]);
}

template <typename T>
cudaError_t launch_dft_sample(const PlaneArgs<T> &a, cudaStream_t s) {
    int n = a.nb * a.nc;
    dft_sample_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// The plane's table of inner phases e^{i w s dt}, s < K, computed in FP64 and rounded
// to the field type once when the plane is added: the folds then spend no FP64
// transcendental per sample and frequency.
template <typename T>
__global__ void dft_phase_kernel(const double *omega, int nfreq, double dt, T *ph) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= DFT_K * nfreq) return;
    const int s = q / nfreq, f = q % nfreq;
    double sn, cs;
    sincos(omega[f] * (double)s * dt, &sn, &cs);
    ph[q] = (T)cs;
    ph[DFT_K * nfreq + q] = (T)sn;
}

template <typename T>
cudaError_t launch_dft_phases(const double *omega, int nfreq, double dt, T *ph, cudaStream_t s) {
    const int n = DFT_K * nfreq;
    dft_phase_kernel<T><<<(n + 255) / 256, 256, 0, s>>>(omega, nfreq, dt, ph);
    return cudaGetLastError();
}

// acc: [4][nfreq][ncell] double2.  step0: step index n of the first sample (it holds
// E at (n+1) dt and H at (n+1/2) dt).  Sample s lies s*dt after the first, so
//   sum_s v_s e^{i w t_s} dt = e^{i w t_0} dt * sum_s v_s e^{i w s dt}:
// the inner K-term sum runs in the field precision T with phases rounded from FP64
// (the plane's table), as does the product with e^{i w t_0} dt; the running sum is
// FP64 (GB300 issues FP64 at a small fraction of the FP32 rate, so the fold keeps
// FP64 to the accumulation).
// The K samples of a thread's cell sit in registers (a partial fold's missing samples
// are zeros, which add nothing), and each group of FC accumulators is loaded before
// any of them is written back.
template <typename T>
__device__ __forceinline__ void fold_body(const T *buf, const T *ph, int nsamp, int ncell, int nfreq,
                                          const double *omega, long long step0, double dt, double2 *acc, long long t) {
    constexpr int FC = 4;
    __shared__ T phr[DFT_K * ML_MAX_FREQS_DEV];
    __shared__ T phi[DFT_K * ML_MAX_FREQS_DEV];
    __shared__ double2 p0[2 * ML_MAX_FREQS_DEV];
    for (int q = threadIdx.x; q < DFT_K * nfreq; q += blockDim.x) {
        phr[q] = ph[q];
        phi[q] = ph[DFT_K * nfreq + q];
    }
    for (int f = threadIdx.x; f < nfreq; f += blockDim.x) {
        double sn, cs;
        sincos(omega[f] * (double)(step0 + 1) * dt, &sn, &cs);
        p0[f] = make_double2(cs * dt, sn * dt);
        sincos(omega[f] * ((double)step0 + 0.5) * dt, &sn, &cs);
        p0[ML_MAX_FREQS_DEV + f] = make_double2(cs * dt, sn * dt);
    }
    __syncthreads();
    if (t >= 4ll * ncell) return;
    const int comp = (int)(t / ncell), cell = (int)(t % ncell);
    const double2 *ph0 = comp < 2 ? p0 : p0 + ML_MAX_FREQS_DEV;
    T v[DFT_K];
#pragma unroll
    for (int s = 0; s < DFT_K; s++) v[s] = s < nsamp ? buf[((long long)s * 4 + comp) * ncell + cell] : T(0);
    double2 *o = acc + (long long)comp * nfreq * ncell + cell;
    for (int f0 = 0; f0 < nfreq; f0 += FC) {
        double2 x[FC];
#pragma unroll
        for (int k = 0; k < FC; k++)
            if (f0 + k < nfreq) x[k] = o[(long long)(f0 + k) * ncell];
#pragma unroll
        for (int k = 0; k < FC; k++) {
            const int f = f0 + k;
            if (f < nfreq) {
                T re = T(0), im = T(0);
#pragma unroll
                for (int s = 0; s < DFT_K; s++) {
                    re += v[s] * phr[s * nfreq + f];
                    im += v[s] * phi[s * nfreq + f];
                }
                const double2 e0 = ph0[f];
                if constexpr (sizeof(T) == 4) {
                    // FP32 fields: the product with e^{i w t_0} dt in FP32 (its rounding is
                    // that of the K-term sum), only the running sum in FP64
                    const float e0x = (float)e0.x, e0y = (float)e0.y;
                    x[k].x += (double)(re * e0x - im * e0y);
                    x[k].y += (double)(re * e0y + im * e0x);
                } else {
                    x[k].x += (double)re * e0.x - (double)im * e0.y;
                    x[k].y += (double)re * e0.y + (double)im * e0.x;
                }
                o[(long long)f * ncell] = x[k];
            }
        }
    }
}

template <typename T>
__global__ void dft_fold_kernel(const T *buf, const T *ph, int nsamp, int ncell, int nfreq, const double *omega,
                                long long step0, double dt, double2 *acc) {
    fold_body(buf, ph, nsamp, ncell, nfreq, omega, step0, dt, acc, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Batched fold: one block per (plane descriptor, 256-entry chunk) work item; the first
// sample's step is the descriptor's base + the device step counter + s_first.
template <typename T>
__global__ void dft_fold_batch_kernel(const FoldBatch<T> b) {
    const int2 wk = b.work[blockIdx.x];
    const FoldDesc<T> d = b.desc[wk.x];
    fold_body(d.buf, d.ph, b.nsamp, d.ncell, d.nfreq, d.omega, d.step_base + *b.boff + b.s_first, b.dt, d.acc,
              (long long)wk.y * blockDim.x + threadIdx.x);
}

template <typename T>
cudaError_t launch_fold_batch(const FoldBatch<T> &b, int nwork, cudaStream_t s) {
    if (nwork == 0 || b.nsamp == 0) return cudaSuccess;
    dft_fold_batch_kernel<T><<<nwork, 256, 0, s>>>(b);
    return cudaGetLastError();
}

__global__ void tick_kernel(long long *c, int add) { *c += add; }

cudaError_t launch_tick(long long *c, int add, cudaStream_t s) {
    tick_kernel<<<1, 1, 0, s>>>(c, add);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dft_fold(const T *buf, int nsamp, int ncell, int nfreq, const double *omega, const T *ph,
                            long long step0, double dt, double2 *acc, cudaStream_t s) {
    if (nsamp == 0) return cudaSuccess;
    long long n = 4ll * ncell;
    int blocks = (int)((n + 255) / 256);
    dft_fold_kernel<T><<<blocks, 256, 0, s>>>(buf, ph, nsamp, ncell, nfreq, omega, step0, dt, acc);
    return cudaGetLastError();
}

// out[f] = sum_cells Re(E_b conj(H_c) - E_c conj(H_b)), one block per frequency,
// fixed-order tree reduction.
__global__ void flux_reduce_kernel(const double2 *acc, int ncell, int nfreq, double *out) {
    __shared__ double red[256];
    const int f = blockIdx.x;
    const double2 *E1 = acc + (0ll * nfreq + f) * ncell;
    const double2 *E2 = acc + (1ll * nfreq + f) * ncell;
    const double2 *H1 = acc + (2ll * nfreq + f) * ncell;
    const double2 *H2 = acc + (3ll * nfreq + f) * ncell;
    double s = 0.0;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
        double2 e1 = E1[c], e2 = E2[c], h1 = H1[c], h2 = H2[c];
        s += (e1.x * h2.x + e1.y * h2.y) - (e2.x * h1.x + e2.y * h1.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0];
}

cudaError_t launch_flux_reduce(const double2 *acc, int ncell, int nfreq, double *out, cudaStream_t s) {
    flux_reduce_kernel<<<nfreq, 256, 0, s>>>(acc, ncell, nfreq, out);
    return cudaGetLastError();
}

#define ML_INST(T)                                                                          \
    template cudaError_t launch_dft_sample<T>(const PlaneArgs<T> &, cudaStream_t);          \
    template cudaError_t launch_dft_fold<T>(const T *, int, int, int, const double *, const T *, long long,    \
                                            double, double2 *, cudaStream_t);                                 \
    template cudaError_t launch_dft_phases<T>(const double *, int, double, T *, cudaStream_t);              \
    template cudaError_t launch_fold_batch<T>(const FoldBatch<T> &, int, cudaStream_t);
ML_INST(float)
ML_INST(double)

}  // namespace ml
