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
// FP64 to the accumulation, once per K steps).
// A thread owns one (component, cell); per group of FC frequencies it stages that
// group's phases in shared memory, loads the FC accumulators, runs the K samples through
// registers SC at a time (a partial fold's missing samples are zeros, which add nothing)
// and writes the accumulators back.
template <typename T>
__device__ __forceinline__ void fold_body(const T *buf, const T *ph, int nsamp, int ncell, int nfreq,
                                          const double *omega, long long step0, double dt, double2 *acc, long long t) {
    constexpr int FC = 8, SC = 8;
    static_assert(DFT_K % SC == 0, "whole sample groups");
    __shared__ __align__(16) T phr[DFT_K][FC];
    __shared__ __align__(16) T phi[DFT_K][FC];
    __shared__ double2 p0[2 * ML_MAX_FREQS_DEV];
    for (int f = threadIdx.x; f < nfreq; f += blockDim.x) {
        double sn, cs;
        sincos(omega[f] * (double)(step0 + 1) * dt, &sn, &cs);
        p0[f] = make_double2(cs * dt, sn * dt);
        sincos(omega[f] * ((double)step0 + 0.5) * dt, &sn, &cs);
        p0[ML_MAX_FREQS_DEV + f] = make_double2(cs * dt, sn * dt);
    }
    const bool act = t < 4ll * ncell;
    const int comp = act ? (int)(t / ncell) : 0, cell = act ? (int)(t % ncell) : 0;
    const double2 *ph0 = comp < 2 ? p0 : p0 + ML_MAX_FREQS_DEV;
    const T *col = buf + (long long)comp * ncell + cell;  // sample s at col[4 s ncell]
    double2 *o = acc + (long long)comp * nfreq * ncell + cell;
    for (int f0 = 0; f0 < nfreq; f0 += FC) {
        __syncthreads();  // the previous group's phases are consumed (p0 is written)
        for (int q = threadIdx.x; q < DFT_K * FC; q += blockDim.x) {
            const int s = q / FC, k = q % FC;
            const bool in = f0 + k < nfreq;
            phr[s][k] = in ? ph[s * nfreq + f0 + k] : T(0);
            phi[s][k] = in ? ph[DFT_K * nfreq + s * nfreq + f0 + k] : T(0);
        }
        __syncthreads();
        if (!act) continue;
        double2 x[FC];
#pragma unroll
        for (int k = 0; k < FC; k++)
            if (f0 + k < nfreq) x[k] = o[(long long)(f0 + k) * ncell];
        T re[FC], im[FC];
#pragma unroll
        for (int k = 0; k < FC; k++) re[k] = im[k] = T(0);
        for (int s0 = 0; s0 < nsamp; s0 += SC) {
            T v[SC];
#pragma unroll
            for (int j = 0; j < SC; j++) v[j] = s0 + j < nsamp ? col[4ll * (s0 + j) * ncell] : T(0);
#pragma unroll
            for (int j = 0; j < SC; j++) {
                T pr[FC], pi[FC];
                if constexpr (sizeof(T) == 4) {  // the group's phases of a sample as 16-byte loads
#pragma unroll
                    for (int k = 0; k < FC; k += 4) {
                        const float4 a = *reinterpret_cast<const float4 *>(&phr[s0 + j][k]);
                        const float4 b = *reinterpret_cast<const float4 *>(&phi[s0 + j][k]);
                        pr[k] = a.x; pr[k + 1] = a.y; pr[k + 2] = a.z; pr[k + 3] = a.w;
                        pi[k] = b.x; pi[k + 1] = b.y; pi[k + 2] = b.z; pi[k + 3] = b.w;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < FC; k++) {
                        pr[k] = phr[s0 + j][k];
                        pi[k] = phi[s0 + j][k];
                    }
                }
#pragma unroll
                for (int k = 0; k < FC; k++) {
                    re[k] += v[j] * pr[k];
                    im[k] += v[j] * pi[k];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < FC; k++) {
            const int f = f0 + k;
            if (f < nfreq) {
                const double2 e0 = ph0[f];
                if constexpr (sizeof(T) == 4) {
                    // FP32 fields: the product with e^{i w t_0} dt in FP32 (its rounding is
                    // that of the K-term sum), only the running sum in FP64
                    const float e0x = (float)e0.x, e0y = (float)e0.y;
                    x[k].x += (double)(re[k] * e0x - im[k] * e0y);
                    x[k].y += (double)(re[k] * e0y + im[k] * e0x);
                } else {
                    x[k].x += (double)re[k] * e0.x - (double)im[k] * e0.y;
                    x[k].y += (double)re[k] * e0.y + (double)im[k] * e0.x;
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

// out[f] = sum_cells Re(E_b conj(H_c) - E_c conj(H_b)) in two fixed-order stages:
// FLUX_NB blocks per frequency each reduce a strided share of the cells into part[f][b]
// with a tree, then one block per frequency adds its FLUX_NB partials with a tree.
__global__ void flux_partial_kernel(const double2 *acc, int ncell, int nfreq, double *part) {
    __shared__ double red[256];
    const int f = blockIdx.y, b = blockIdx.x;
    const double2 *E1 = acc + (0ll * nfreq + f) * ncell;
    const double2 *E2 = acc + (1ll * nfreq + f) * ncell;
    const double2 *H1 = acc + (2ll * nfreq + f) * ncell;
    const double2 *H2 = acc + (3ll * nfreq + f) * ncell;
    double s = 0.0;
    for (int c = b * blockDim.x + threadIdx.x; c < ncell; c += FLUX_NB * blockDim.x) {
        double2 e1 = E1[c], e2 = E2[c], h1 = H1[c], h2 = H2[c];
        s += (e1.x * h2.x + e1.y * h2.y) - (e2.x * h1.x + e2.y * h1.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[f * FLUX_NB + b] = red[0];
}

__global__ void flux_final_kernel(const double *part, double *out) {
    __shared__ double red[FLUX_NB];
    const int f = blockIdx.x;
    red[threadIdx.x] = part[f * FLUX_NB + threadIdx.x];
    __syncthreads();
    for (int o = FLUX_NB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = red[0];
}

cudaError_t launch_flux_reduce(const double2 *acc, int ncell, int nfreq, double *part, double *out, cudaStream_t s) {
    flux_partial_kernel<<<dim3(FLUX_NB, nfreq), 256, 0, s>>>(acc, ncell, nfreq, part);
    flux_final_kernel<<<nfreq, FLUX_NB, 0, s>>>(part, out);
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
