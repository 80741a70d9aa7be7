// K2: one warp per molecule, once per time step.
//   1. regularised field Etilde_m^c = gamma_m sum_window E^c kappa_m^c
//      (Eq. E_regu_Emi): the sum of the molecule's gather partials (one per box
//      block its window touches, written by the gather kernel), in list order;
//   2. density-matrix step under H0 - Etilde . mu held over dt (Eq.
//      von-Neumann-tls): closed-form 2x2 exponential, or classic RK4 substeps of
//      the GKSL equation with ladder decay and pure dephasing written element-wise;
//   3. mudot = (Tr rho' mu - Tr rho mu) / dt (Eq. dipole_derivative) and the
//      current amplitude gamma * mudot consumed by the field pass (Eq. J_mol);
//   4. FP64 running sum of Tr(rho H0) for the time-averaged molecular energy.
// K3 (setup): separable, normalised 1D Gaussian weights per molecule, axis and
// staggering, folded onto one period on periodic axes.
#include <algorithm>

#include "ml_internal.cuh"

namespace ml {

template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <typename T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.re, -a.im}; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ long long fidx(int px, long long plane, int i, int j, int k) {
    return (long long)(k + 1) * plane + (long long)(j + 1) * px + (i + XO);
}

constexpr int MOL_WARPS = 4;
constexpr int MOL_MIN_BLOCKS = 6;
constexpr int MU_MIN_BLOCKS = 3;        // FP32 thread-per-molecule kernel: resident blocks per SM the register budget is cut for
constexpr int MU_MIN_BLOCKS_EXACT = 4;  // the same, every molecule on the exact 2x2 step

template <typename T>
struct MolShared {
    cx<T> H[MOL_WARPS][MAXLEV * MAXLEV];
    cx<T> S[MOL_WARPS][2][MAXLEV * MAXLEV];
    T W[MOL_WARPS][NW];  // the molecule's 1D kernel weights (window form)
};

// Regularised-field sums of molecule m straight from the field (Eq. E_regu_Emi without
// gamma): g_c = sum_window wx wy wz E^c over the canonical window (start win, folded
// length wf; periodic axes wrap), component c sampled half a cell along c.  Lane
// (dx = lane & 15, row parity = lane >> 4) sums its x column over the rows of its
// parity and the planes in fixed order; the xor tree then adds the lanes.
template <typename T>
__device__ __forceinline__ void window_gather(const MolArgs<T> &a, const int m, const int cm, const T *sw, T (&g)[3]) {
    const int lane = threadIdx.x & 31, dx = lane & 15, py = lane >> 4;
    const int wfm = a.wf[m];
    const int Wx = wfm & 0xff, Wy = (wfm >> 8) & 0xff, Wz = (wfm >> 16) & 0xff;
    const int x0 = a.win[3 * m], y0 = a.win[3 * m + 1], z0 = a.win[3 * m + 2];
    int x = x0 + dx;
    if (x >= a.nx) x -= a.nx;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        T t = T(0);
        if (((cm >> c) & 1) && dx < Wx) {
            const T *E = a.E[c] + x + XO;
            const T *wy = sw + (2 + (c == 1 ? 1 : 0)) * WMAX, *wz = sw + (4 + (c == 2 ? 1 : 0)) * WMAX;
            // row offsets of this lane's rows (fixed bound, predicated: all loads of a
            // plane are in flight together)
            long long roff[WMAX / 2];
            T wyv[WMAX / 2];
#pragma unroll
            for (int q = 0; q < WMAX / 2; q++) {
                const int dy = py + 2 * q;
                int y = y0 + dy;
                if (y >= a.ny) y -= a.ny;
                roff[q] = (long long)(y + 1) * a.px;
                wyv[q] = dy < Wy ? wy[dy] : T(0);
            }
            for (int dz = 0; dz < Wz; dz += 2) {
                T u0 = T(0), u1 = T(0);
                int z = z0 + dz;
                if (z >= a.nz) z -= a.nz;
                int z1 = z + 1;
                if (z1 >= a.nz) z1 -= a.nz;
                const bool two = dz + 1 < Wz;
                const T *Ez = E + (long long)(z + 1) * a.plane, *Ez1 = E + (long long)(z1 + 1) * a.plane;
                T v0[WMAX / 2], v1[WMAX / 2];
#pragma unroll
                for (int q = 0; q < WMAX / 2; q++) {
                    const bool in = py + 2 * q < Wy;
                    v0[q] = in ? Ez[roff[q]] : T(0);
                    v1[q] = (in && two) ? Ez1[roff[q]] : T(0);
                }
#pragma unroll
                for (int q = 0; q < WMAX / 2; q++) {
                    u0 += wyv[q] * v0[q];
                    u1 += wyv[q] * v1[q];
                }
                t += wz[dz] * u0;
                if (two) t += wz[dz + 1] * u1;
            }
            t *= sw[(c == 0 ? 1 : 0) * WMAX + dx];
        }
        g[c] = ((cm >> c) & 1) ? warp_sum(t) : T(0);
    }
}

// FP32 form of window_gather for a window that wraps on no axis and whose x extent,
// widened to whole 16-byte groups, is at most 16 values: every padded row starts on a
// 128-byte boundary, so the group starting at x0 & ~3 is aligned.  Lane = 4 * row +
// group; rows rr and rr + 8.  Per plane a lane issues one 16-byte load per row, folds
// the four values with its x weights (zero outside the window) and accumulates wz times
// that; the y weights are applied at the end and the xor tree adds the lanes.  The
// rows and groups past the window are never loaded.  Returns false when the window
// does not qualify (the caller then takes window_gather).
__device__ __forceinline__ bool window_gather_vec(const MolArgs<float> &a, const int cm, const int wfm, const int x0,
                                                  const int y0, const int z0, const float *sw, float (&g)[3]) {
    const int Wx = wfm & 0xff, Wy = (wfm >> 8) & 0xff, Wz = (wfm >> 16) & 0xff;
    const int xa = x0 & ~3, sx = x0 - xa;
    if (sx + Wx > 16 || x0 + Wx > a.nx || y0 + Wy > a.ny || z0 + Wz > a.nz) return false;
    const int lane = threadIdx.x & 31, qd = lane & 3, rr = lane >> 2;
    const bool in0 = rr < Wy, in1 = rr + 8 < Wy;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float t = 0.f;
        if ((cm >> c) & 1) {
            const float *wx = sw + (c == 0 ? 1 : 0) * WMAX, *wy = sw + (2 + (c == 1 ? 1 : 0)) * WMAX,
                        *wz = sw + (4 + (c == 2 ? 1 : 0)) * WMAX;
            float wxk[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int d = 4 * qd + k - sx;
                wxk[k] = (unsigned)d < (unsigned)Wx ? wx[d] : 0.f;
            }
            const float *p0 = a.E[c] + (long long)(z0 + 1) * a.plane + (long long)(y0 + rr + 1) * a.px + XO + xa + 4 * qd;
            const float *p1 = p0 + 8ll * a.px;
            float acc0 = 0.f, acc1 = 0.f;
            for (int dz = 0; dz < Wz; dz += 4) {
                float4 v0[4], v1[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const bool pz = dz + k < Wz;
                    const long long o = (long long)k * a.plane;
                    v0[k] = (pz && in0) ? __ldg(reinterpret_cast<const float4 *>(p0 + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    v1[k] = (pz && in1) ? __ldg(reinterpret_cast<const float4 *>(p1 + o)) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const float w = dz + k < Wz ? wz[dz + k] : 0.f;
                    acc0 += w * (wxk[0] * v0[k].x + wxk[1] * v0[k].y + wxk[2] * v0[k].z + wxk[3] * v0[k].w);
                    acc1 += w * (wxk[0] * v1[k].x + wxk[1] * v1[k].y + wxk[2] * v1[k].z + wxk[3] * v1[k].w);
                }
                p0 += 4 * a.plane;
                p1 += 4 * a.plane;
            }
            t = (in0 ? wy[rr] : 0.f) * acc0 + (in1 ? wy[rr + 8] : 0.f) * acc1;
        }
        g[c] = ((cm >> c) & 1) ? warp_sum(t) : 0.f;
    }
    return true;
}

// The uniform-field source's field at molecule m before gamma_m: Eu, or the laser's
// plane wave on |u| < W.  With FP64 fields u = (z_m - xi0) - t is FP64.  With FP32 fields
// both z_m - xi0 and t arrive as float pairs (hi + lo, the pair rounded from FP64), and u
// is their difference by Knuth's two-sum of the high parts plus the low parts: the same
// u to about 2^-48 of |z_m - xi0| + |t|, without FP64 arithmetic, which GB300 issues at
// a small fraction of the FP32 rate.
template <typename T>
__device__ __forceinline__ void uniform_field(const MolArgs<T> &a, const int m, T (&E)[3]) {
    if (!a.laser) {
#pragma unroll
        for (int c = 0; c < 3; c++) E[c] = a.Eu[c];
        return;
    }
    T uf;
    bool in;
    if constexpr (sizeof(T) == 8) {
        const double u = (a.zpos[m] - a.lxi0) - (double)(*a.lbase + a.lstep) * a.ldt;
        in = fabs(u) < a.lW;
        uf = u;
    } else {
        const float2 z = a.lzr[m], t = a.ltt[a.lstep];
        const float s = z.x - t.x, v = s - z.x;
        const float err = (z.x - (s - v)) + (-t.x - v);
        uf = s + (err + (z.y - t.y));
        in = fabsf(uf) < a.lW;
    }
    T f = T(0);
    if (in) {
        const T cw = cos(T(1.5707963267948966) * uf / a.lW);
        f = a.lE0 * cw * cw * cos(a.lk * uf + a.lphase);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) E[c] = f * a.lpol[c];
}

// GKSL right-hand side for element (j,l) of rho given in S (n x n), H in Hs.
template <typename T>
__device__ __forceinline__ cx<T> rhs_elem(int n, int j, int l, const cx<T> *S, const cx<T> *Hs, T decay, T deph) {
    cx<T> acc = {T(0), T(0)};
    for (int p = 0; p < n; p++) {
        cx<T> a = cmul(Hs[j * n + p], S[p * n + l]);
        cx<T> b = cmul(S[j * n + p], Hs[p * n + l]);
        acc.re += a.re - b.re;
        acc.im += a.im - b.im;
    }
    // -i * acc
    cx<T> out = {acc.im, -acc.re};
    const cx<T> r = S[j * n + l];
    if (decay != T(0)) {
        T f = T(0.5) * decay * (T(j >= 1) + T(l >= 1));
        out.re -= f * r.re;
        out.im -= f * r.im;
        if (j == l && j + 1 < n) out.re += decay * S[(j + 1) * n + (j + 1)].re;
    }
    if (deph != T(0) && j != l) {
        out.re -= deph * r.re;
        out.im -= deph * r.im;
    }
    return out;
}

// SRC: where the regularised field comes from.  SRC_WINDOW: the warp gathers its own
// window from E (window_gather); SRC_UNIFORM: one field for every molecule (a.Eu, times
// gamma_m), as in the single-mode cavity, and the warp also writes gamma_m <mu> of the
// new state.
constexpr int SRC_WINDOW = 1, SRC_UNIFORM = 2;
template <typename T, int SRC, bool N2>
__device__ __forceinline__ void molecule_body(const MolArgs<T> &a, const int m0) {
    static_assert(SRC == SRC_WINDOW || SRC == SRC_UNIFORM, "unknown field source");
    __shared__ MolShared<T> sh;
    const int lane = threadIdx.x & 31;
    const int wl = threadIdx.x >> 5;
    const int m = m0 + wl;
    if (m >= a.nmol) return;  // whole warp leaves together

    // ---- 0. every load of this molecule's data, issued before any is used.  N2: every
    // molecule has two levels at pool offset 4 m, so no load waits for another (the
    // dipole of an absent component is zero in the pool and is loaded as such) and the
    // Lindblad right-hand side is unrolled for n = 2.
    const int n = N2 ? 2 : a.nlev[m];
    const int nn = n * n;
    const long long o = N2 ? 4ll * m : a.off[m];
    const int cm = a.cmask[m];
    const int kind = a.kind[m];
    const T gam = a.gamma[m];
    const double e_old = lane == 0 ? a.energy[m] : 0.0;
    // the kernel window and its weights (SRC_WINDOW)
    static_assert(NW == 96, "three weights per lane");
    int wfm = 0, x0 = 0, y0 = 0, z0 = 0;
    T wreg[3];
    if (SRC == SRC_WINDOW) {
#pragma unroll
        for (int q = 0; q < 3; q++) wreg[q] = a.w[(long long)m * NW + lane + 32 * q];
        wfm = a.wf[m];
        x0 = a.win[3 * m];
        y0 = a.win[3 * m + 1];
        z0 = a.win[3 * m + 2];
    }
    // lane owns density-matrix elements e = lane and e = lane + 32 (row-major n x n)
    cx<T> r0[2], h0[2], mu[3][2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int e = lane + 32 * q;
        const bool in = e < nn;
        r0[q] = in ? a.rho[o + e] : cx<T>{T(0), T(0)};
        h0[q] = in ? a.H0[o + e] : cx<T>{T(0), T(0)};
#pragma unroll
        for (int c = 0; c < 3; c++)
            mu[c][q] = (in && (N2 || ((cm >> c) & 1))) ? a.mu[c * a.pool + o + e] : cx<T>{T(0), T(0)};
    }
    if (SRC == SRC_WINDOW) {
#pragma unroll
        for (int q = 0; q < 3; q++) sh.W[wl][lane + 32 * q] = wreg[q];
    }
    __syncwarp();

    // ---- programmatic dependence: everything above is this molecule's own state.  When
    // the kernel is launched as the previous field pass's dependent, the field (or the
    // gather partials) is read only after that pass has completed, and the current
    // kernel is released only then.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // ---- 1. regularised field
    T Et[3];
    if (SRC == SRC_UNIFORM) {
        uniform_field(a, m, Et);
#pragma unroll
        for (int c = 0; c < 3; c++) Et[c] *= gam;
    } else {
        const T *sw = sh.W[wl];
        T g[3];
        bool done = false;
        if constexpr (sizeof(T) == 4) done = window_gather_vec(a, cm, wfm, x0, y0, z0, sw, g);
        if (!done) window_gather(a, m, cm, sw, g);
#pragma unroll
        for (int c = 0; c < 3; c++) Et[c] = gam * g[c];
    }

    // ---- 2. H = H0 - Etilde . mu and <mu> before the step.  For Hermitian
    // operators Re Tr(rho A) = sum_jl Re(rho_jl conj(A_jl)): own elements only.
    cx<T> *Hs = sh.H[wl];
    T mu0[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int e = lane + 32 * q;
        if (e < nn) {
            cx<T> h = h0[q];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                h.re -= Et[c] * mu[c][q].re;
                h.im -= Et[c] * mu[c][q].im;
                mu0[c] += r0[q].re * mu[c][q].re + r0[q].im * mu[c][q].im;
            }
            Hs[e] = h;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; c++) mu0[c] = ((cm >> c) & 1) ? warp_sum(mu0[c]) : T(0);
    __syncwarp();

    // ---- 3. density-matrix step over dt with the field held
    cx<T> r1[2] = {r0[0], r0[1]};
    // RK4: the change of the own elements over the step, summed from the substeps'
    // increments.  d<mu>/dt is Re Tr(drho mu)/dt (Eq. dipole_derivative): the same
    // quantity as the difference of the two traces, without the cancellation of the
    // diagonal terms of mu in FP32.
    cx<T> dr[2] = {{T(0), T(0)}, {T(0), T(0)}};
    const bool incr = kind != 0;
    if (kind == 0) {
        // exact exponential of a 2x2 Hermitian H:
        // U = e^{-i hbar dt}[cos(W dt) - i sin(W dt)/W (H - hbar)], the phase cancels in U rho U^+
        // gather rho (elements 0..3 live on lanes 0..3) into shared memory first
        if (lane < 4) sh.S[wl][0][lane] = r0[0];
        __syncwarp();
        if (lane == 0) {
            const T dt = a.dt;
            const T ha = Hs[0].re, hd = Hs[3].re;
            const cx<T> b = Hs[1];
            const T z = T(0.5) * (ha - hd);
            const T W = sqrt(z * z + b.re * b.re + b.im * b.im);
            const T cw = cos(W * dt);
            const T sw = W > T(0) ? sin(W * dt) / W : dt;
            cx<T> U[4];
            U[0] = {cw, -sw * z};
            U[1] = {sw * b.im, -sw * b.re};   // -i sw b
            U[2] = {-sw * b.im, -sw * b.re};  // -i sw conj(b)
            U[3] = {cw, sw * z};
            cx<T> R[4];
            for (int e = 0; e < 4; e++) R[e] = sh.S[wl][0][e];
            cx<T> TT[4], out[4];
            for (int p = 0; p < 2; p++)
                for (int q = 0; q < 2; q++)
                    TT[p * 2 + q] = cadd(cmul(U[p * 2 + 0], R[0 * 2 + q]), cmul(U[p * 2 + 1], R[1 * 2 + q]));
            for (int p = 0; p < 2; p++)
                for (int q = 0; q < 2; q++)
                    out[p * 2 + q] =
                        cadd(cmul(TT[p * 2 + 0], cconj(U[q * 2 + 0])), cmul(TT[p * 2 + 1], cconj(U[q * 2 + 1])));
            for (int e = 0; e < 4; e++) sh.S[wl][1][e] = out[e];
        }
        __syncwarp();
        if (lane < 4) r1[0] = sh.S[wl][1][lane];
    } else {
        const int ns = a.nsub[m];
        const T h = a.dt / T(ns);
        const T decay = a.decay[m], deph = a.dephase[m];
        const int e0 = lane, e1 = lane + 32;
        const int j0 = e0 / n, l0 = e0 - j0 * n, j1 = e1 / n, l1 = e1 - j1 * n;
        for (int sstep = 0; sstep < ns; sstep++) {
            cx<T> base[2] = {r1[0], r1[1]};
            cx<T> acc[2] = {{T(0), T(0)}, {T(0), T(0)}};
            if (e0 < nn) sh.S[wl][0][e0] = base[0];
            if (e1 < nn) sh.S[wl][0][e1] = base[1];
            __syncwarp();
            int sb = 0;
#pragma unroll 1
            for (int st = 0; st < 4; st++) {
                const T wgt = (st == 0 || st == 3) ? T(1) : T(2);
                const T cn = (st < 2) ? T(0.5) : T(1);
                cx<T> f[2];
                if (e0 < nn) {
                    f[0] = rhs_elem(n, j0, l0, sh.S[wl][sb], Hs, decay, deph);
                    acc[0].re += wgt * f[0].re;
                    acc[0].im += wgt * f[0].im;
                }
                if (e1 < nn) {
                    f[1] = rhs_elem(n, j1, l1, sh.S[wl][sb], Hs, decay, deph);
                    acc[1].re += wgt * f[1].re;
                    acc[1].im += wgt * f[1].im;
                }
                if (st < 3) {
                    if (e0 < nn) sh.S[wl][sb ^ 1][e0] = {base[0].re + cn * h * f[0].re, base[0].im + cn * h * f[0].im};
                    if (e1 < nn) sh.S[wl][sb ^ 1][e1] = {base[1].re + cn * h * f[1].re, base[1].im + cn * h * f[1].im};
                    sb ^= 1;
                    __syncwarp();
                }
            }
            for (int q = 0; q < 2; q++) {
                const T ur = h / T(6) * acc[q].re, ui = h / T(6) * acc[q].im;
                r1[q].re = base[q].re + ur;
                r1[q].im = base[q].im + ui;
                dr[q].re += ur;
                dr[q].im += ui;
            }
            __syncwarp();
        }
    }
    // ---- 4. <mu> after, mudot, current amplitude, energy
    T mu1[3] = {T(0), T(0), T(0)};
    T dmu[3] = {T(0), T(0), T(0)};
    T en = T(0);
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int e = lane + 32 * q;
        if (e < nn) {
            a.rho[o + e] = r1[q];
            if (a.pop_sink && e % (n + 1) == 0)  // diagonal element (j, j), j = e / (n + 1)
                a.pop_sink[a.pop_slot + (long long)m * MAXLEV + e / (n + 1)] = (double)r1[q].re;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                mu1[c] += r1[q].re * mu[c][q].re + r1[q].im * mu[c][q].im;
                dmu[c] += dr[q].re * mu[c][q].re + dr[q].im * mu[c][q].im;
            }
            en += r1[q].re * h0[q].re + r1[q].im * h0[q].im;
        }
    }
    en = warp_sum(en);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        mu1[c] = ((cm >> c) & 1) ? warp_sum(mu1[c]) : T(0);
        if (incr) dmu[c] = ((cm >> c) & 1) ? warp_sum(dmu[c]) : T(0);
    }
    if (lane == 0) {
        bool bad = false;
        for (int c = 0; c < 3; c++) {
            const T md = (incr ? dmu[c] : mu1[c] - mu0[c]) / a.dt;
            a.Et[3 * m + c] = Et[c];
            a.mudot[3 * m + c] = md;
            a.c[3 * m + c] = gam * md;
            if (SRC == SRC_UNIFORM) a.gmu[3 * m + c] = gam * mu1[c];
            if (!isfinite(Et[c]) || !isfinite(md)) bad = true;
        }
        a.energy[m] = e_old + (double)en;
        if (bad) atomicCAS(a.status, 0, 6);
    }
}

// The kernel may be launched as the previous field pass's programmatic dependent, and
// the current kernel as this one's: molecule_body waits for the field pass before it
// reads the field and releases the current kernel after that wait (the current kernel
// waits for this kernel's completion before it reads the amplitudes).
// N2: every molecule has two levels (see molecule_body).
template <typename T, bool N2>
__global__ void __launch_bounds__(MOL_WARPS * 32, sizeof(T) == 4 ? MOL_MIN_BLOCKS : 1) molecule_kernel(const MolArgs<T> a) {
    molecule_body<T, SRC_WINDOW, N2>(a, (int)blockIdx.x * MOL_WARPS);
}

// ------------------------------------------------------------------ packed molecules
// Grids with multilevel molecules: one warp per work item of up to pack_per_warp(n)
// molecules of one kind, level count n and substep count (sorted on the host).  The
// warp gathers each molecule's regularised field in turn (Eq. E_regu_Emi, as in
// molecule_body), then steps all of them at once: the density matrix and the RK4 stages
// are Hermitian, so a molecule's group of lanes holds only its upper-triangle elements
// (lane u of the group owns element u of the row-major upper triangle, and u + 32 too
// for n = 8) and writes each new element to both halves of the shared matrix; the GKSL
// right-hand side is unrolled for the compile-time n.  d<mu>/dt is Re Tr(drho mu)/dt
// with drho the step's increment (Eq. dipole_derivative).
template <typename T>
struct PackShared {
    cx<T> S[MOL_WARPS][2][64];  // per molecule q of the warp: matrix at q * n * n
    cx<T> H[MOL_WARPS][64];
    T W[MOL_WARPS][NW];
    T Et[MOL_WARPS][8][3];
    cx<T> K[MOL_WARPS][2][4][32];  // per lane and slot: H0 and the three dipole elements,
                                   // kept for the outputs while the RK4 stages run
};

// (j, l), j <= l, of upper-triangle element u (row-major) of an n x n matrix
template <int N>
__device__ __forceinline__ void upper_index(int u, int &j, int &l) {
    j = 0;
#pragma unroll
    for (int q = 0; q < N; q++)
        if (j == q && u >= N - q) {
            u -= N - q;
            j = q + 1;
        }
    l = j + u;
}

// GKSL right-hand side of element (j, l) (the rhs_elem formula, n fixed at compile time)
template <typename T, int N>
__device__ __forceinline__ cx<T> rhs_fixed(int j, int l, const cx<T> *S, const cx<T> *H, T decay, T deph) {
    cx<T> acc = {T(0), T(0)};
#pragma unroll
    for (int p = 0; p < N; p++) {
        const cx<T> x = cmul(H[j * N + p], S[p * N + l]);
        const cx<T> y = cmul(S[j * N + p], H[p * N + l]);
        acc.re += x.re - y.re;
        acc.im += x.im - y.im;
    }
    cx<T> out = {acc.im, -acc.re};
    const cx<T> r = S[j * N + l];
    if (decay != T(0)) {
        const T f = T(0.5) * decay * (T(j >= 1) + T(l >= 1));
        out.re -= f * r.re;
        out.im -= f * r.im;
        if (j == l && j + 1 < N) out.re += decay * S[(j + 1) * N + (j + 1)].re;
    }
    if (deph != T(0) && j != l) {
        out.re -= deph * r.re;
        out.im -= deph * r.im;
    }
    return out;
}

// sum over the lanes of a group of G (a power of two <= 32; 64: the whole warp)
template <typename T, int G>
__device__ __forceinline__ T group_sum(T v) {
    constexpr int W = G > 32 ? 32 : G;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int N, bool EXACT>
__device__ __forceinline__ void packed_body(const MolArgs<T> &a, const int4 item, PackShared<T> &sh, const int wl) {
    constexpr int G = pack_group(N), NN = N * N, NE = N * (N + 1) / 2, SL = G > 32 ? 2 : 1;
    constexpr int GL = G > 32 ? 32 : G;  // lanes per group
    const int lane = threadIdx.x & 31;
    const int q = lane / GL, u0 = lane % GL;
    const int cnt = item.y;
    const bool live = q < cnt;
    const int m = a.order[item.x + (live ? q : 0)];
    int jj[SL], ll[SL];
    bool own[SL];
#pragma unroll
    for (int s = 0; s < SL; s++) {
        const int u = u0 + 32 * s;
        own[s] = live && u < NE;
        upper_index<N>(own[s] ? u : 0, jj[s], ll[s]);
    }
    // ---- this molecule's own elements and parameters, loaded before the dependence wait
    const long long o = a.off[m];
    const int cm = a.cmask[m];
    const T gam = a.gamma[m];
    const T decay = EXACT ? T(0) : a.decay[m], deph = EXACT ? T(0) : a.dephase[m];
    const double e_old = (live && u0 == 0) ? a.energy[m] : 0.0;
    cx<T> r0[SL], h0[SL], mu[3][SL];
#pragma unroll
    for (int s = 0; s < SL; s++) {
        const long long e = o + jj[s] * N + ll[s];
        r0[s] = own[s] ? a.rho[e] : cx<T>{T(0), T(0)};
        h0[s] = own[s] ? a.H0[e] : cx<T>{T(0), T(0)};
#pragma unroll
        for (int c = 0; c < 3; c++) mu[c][s] = (own[s] && ((cm >> c) & 1)) ? a.mu[c * a.pool + e] : cx<T>{T(0), T(0)};
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // ---- 1. regularised fields, one molecule of the item after the other (whole warp;
    // a separate gather kernel with many more windows in flight measured slower overall:
    // 0.250 vs 0.239 ms per step on the 512 x 512 x 384 ensemble)
    for (int qq = 0; qq < cnt; qq++) {
        const int mq = a.order[item.x + qq];
        const T w0 = a.w[(long long)mq * NW + lane], w1 = a.w[(long long)mq * NW + lane + 32],
                w2 = a.w[(long long)mq * NW + lane + 64];
        const int wfm = a.wf[mq], x0 = a.win[3 * mq], y0 = a.win[3 * mq + 1], z0 = a.win[3 * mq + 2];
        const int cmq = a.cmask[mq];
        __syncwarp();
        sh.W[wl][lane] = w0;
        sh.W[wl][lane + 32] = w1;
        sh.W[wl][lane + 64] = w2;
        __syncwarp();
        T g[3];
        bool done = false;
        if constexpr (sizeof(T) == 4) done = window_gather_vec(a, cmq, wfm, x0, y0, z0, sh.W[wl], g);
        if (!done) window_gather(a, mq, cmq, sh.W[wl], g);
        if (lane == 0) {
            const T gq = a.gamma[mq];
#pragma unroll
            for (int c = 0; c < 3; c++) sh.Et[wl][qq][c] = gq * g[c];
        }
    }
    __syncwarp();
    T Et[3];
#pragma unroll
    for (int c = 0; c < 3; c++) Et[c] = live ? sh.Et[wl][q][c] : T(0);

    // ---- 2. H = H0 - Et . mu and S = rho, both halves of each matrix
    cx<T> *Hs = sh.H[wl] + q * NN;
    cx<T> *S0 = sh.S[wl][0] + q * NN, *S1 = sh.S[wl][1] + q * NN;
#pragma unroll
    for (int s = 0; s < SL; s++) {
        sh.K[wl][s][0][lane] = h0[s];
#pragma unroll
        for (int c = 0; c < 3; c++) sh.K[wl][s][1 + c][lane] = mu[c][s];
    }
#pragma unroll
    for (int s = 0; s < SL; s++)
        if (own[s]) {
            cx<T> h = h0[s];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                h.re -= Et[c] * mu[c][s].re;
                h.im -= Et[c] * mu[c][s].im;
            }
            const int j = jj[s], l = ll[s];
            Hs[j * N + l] = h;
            Hs[l * N + j] = cconj(h);
            S0[j * N + l] = r0[s];
            S0[l * N + j] = cconj(r0[s]);
        }
    __syncwarp();

    // ---- 3. the step
    cx<T> r1[SL], dr[SL];
    if constexpr (EXACT) {
        // U = cos(W dt) - i sin(W dt)/W (H - tr H / 2): the exact propagator of the held
        // 2x2 Hamiltonian (its phase cancels); rho' = U rho U^+; for d<mu>/dt the increment
        // A rho + rho A^+ + A rho A^+ with A = U - 1 (cos(W dt) - 1 = -2 sin^2(W dt / 2))
        const T dt = a.dt;
        const T z = T(0.5) * (Hs[0].re - Hs[3].re);
        const cx<T> b = Hs[1];
        const T W = sqrt(z * z + b.re * b.re + b.im * b.im);
        const T sh2 = sin(T(0.5) * W * dt);
        const T cm1 = T(-2) * sh2 * sh2;
        const T sw = W > T(0) ? sin(W * dt) / W : dt;
        const cx<T> a00 = {cm1, -sw * z}, a01 = {sw * b.im, -sw * b.re}, a10 = {-sw * b.im, -sw * b.re},
                    a11 = {cm1, sw * z};
        const int j = jj[0], l = ll[0];
        // rows j and l of A and of U = 1 + A, and the columns l of rho (no indexed arrays)
        const cx<T> aj0 = j ? a10 : a00, aj1 = j ? a11 : a01, al0 = l ? a10 : a00, al1 = l ? a11 : a01;
        const cx<T> uj0 = {aj0.re + T(j == 0), aj0.im}, uj1 = {aj1.re + T(j == 1), aj1.im};
        const cx<T> ul0 = {al0.re + T(l == 0), al0.im}, ul1 = {al1.re + T(l == 1), al1.im};
        const cx<T> R00 = S0[0], R01 = S0[1], R10 = S0[2], R11 = S0[3];
        const cx<T> Rj0 = j ? R10 : R00, Rj1 = j ? R11 : R01;  // row j of rho
        const cx<T> R0l = l ? R01 : R00, R1l = l ? R11 : R10;  // column l of rho
        // (X rho Y^+)_jl for rows x0, x1 of X and y0, y1 of Y
        auto sand = [&](cx<T> x0, cx<T> x1, cx<T> y0, cx<T> y1) {
            const cx<T> t0 = cadd(cmul(x0, R00), cmul(x1, R10)), t1 = cadd(cmul(x0, R01), cmul(x1, R11));
            return cadd(cmul(t0, cconj(y0)), cmul(t1, cconj(y1)));
        };
        r1[0] = sand(uj0, uj1, ul0, ul1);
        cx<T> d = sand(aj0, aj1, al0, al1);
        d = cadd(d, cadd(cmul(aj0, R0l), cmul(aj1, R1l)));                  // (A rho)_jl
        d = cadd(d, cadd(cmul(Rj0, cconj(al0)), cmul(Rj1, cconj(al1))));    // (rho A^+)_jl
        dr[0] = d;
    } else {
        const int ns = item.w >> 4;
        const T h = a.dt / T(ns);
#pragma unroll
        for (int s = 0; s < SL; s++) {
            r1[s] = r0[s];
            dr[s] = {T(0), T(0)};
        }
        for (int sstep = 0; sstep < ns; sstep++) {
            cx<T> base[SL], acc[SL];
#pragma unroll
            for (int s = 0; s < SL; s++) {
                base[s] = r1[s];
                acc[s] = {T(0), T(0)};
            }
            const cx<T> *Sc = S0;
            cx<T> *Sn = S1;
#pragma unroll
            for (int st = 0; st < 4; st++) {
                const T wgt = (st == 0 || st == 3) ? T(1) : T(2);
                const T cn = (st < 2) ? T(0.5) : T(1);
                cx<T> f[SL];
#pragma unroll
                for (int s = 0; s < SL; s++)
                    if (own[s]) {
                        f[s] = rhs_fixed<T, N>(jj[s], ll[s], Sc, Hs, decay, deph);
                        acc[s].re += wgt * f[s].re;
                        acc[s].im += wgt * f[s].im;
                    }
                if (st < 3) {
#pragma unroll
                    for (int s = 0; s < SL; s++)
                        if (own[s]) {
                            const cx<T> v = {base[s].re + cn * h * f[s].re, base[s].im + cn * h * f[s].im};
                            Sn[jj[s] * N + ll[s]] = v;
                            Sn[ll[s] * N + jj[s]] = cconj(v);
                        }
                    __syncwarp();
                    const cx<T> *t = Sc;
                    Sc = Sn;
                    Sn = const_cast<cx<T> *>(t);
                }
            }
#pragma unroll
            for (int s = 0; s < SL; s++) {
                const T ur = h / T(6) * acc[s].re, ui = h / T(6) * acc[s].im;
                r1[s] = {base[s].re + ur, base[s].im + ui};
                dr[s].re += ur;
                dr[s].im += ui;
            }
            if (sstep + 1 < ns) {
                __syncwarp();  // every lane is done reading the stage matrices
#pragma unroll
                for (int s = 0; s < SL; s++)
                    if (own[s]) {
                        S0[jj[s] * N + ll[s]] = r1[s];
                        S0[ll[s] * N + jj[s]] = cconj(r1[s]);
                    }
                __syncwarp();
            }
        }
    }

    // ---- 4. outputs: rho (both halves), d<mu>/dt, current amplitude, energy sum
    T dmu[3] = {T(0), T(0), T(0)};
    T en = T(0);
#pragma unroll
    for (int s = 0; s < SL; s++)
        if (own[s]) {
            h0[s] = sh.K[wl][s][0][lane];
#pragma unroll
            for (int c = 0; c < 3; c++) mu[c][s] = sh.K[wl][s][1 + c][lane];
            const int j = jj[s], l = ll[s];
            const T wt = j == l ? T(1) : T(2);  // Re Tr(X A) over both halves of Hermitian X, A
            a.rho[o + j * N + l] = r1[s];
            if (j != l) a.rho[o + l * N + j] = cconj(r1[s]);
            else if (a.pop_sink) a.pop_sink[a.pop_slot + (long long)m * MAXLEV + j] = (double)r1[s].re;
#pragma unroll
            for (int c = 0; c < 3; c++) dmu[c] += wt * (dr[s].re * mu[c][s].re + dr[s].im * mu[c][s].im);
            en += wt * (r1[s].re * h0[s].re + r1[s].im * h0[s].im);
        }
    en = group_sum<T, G>(en);
#pragma unroll
    for (int c = 0; c < 3; c++) dmu[c] = ((cm >> c) & 1) ? group_sum<T, G>(dmu[c]) : T(0);
    if (live && u0 == 0) {
        bool bad = false;
        for (int c = 0; c < 3; c++) {
            const T md = dmu[c] / a.dt;
            a.Et[3 * m + c] = Et[c];
            a.mudot[3 * m + c] = md;
            a.c[3 * m + c] = gam * md;
            if (!isfinite(Et[c]) || !isfinite(md)) bad = true;
        }
        a.energy[m] = e_old + (double)en;
        if (bad) atomicCAS(a.status, 0, 6);
    }
}

// Work item `it` of the packed form (one warp), dispatched on its kind and level count.
template <typename T>
__device__ __forceinline__ void packed_item(const MolArgs<T> &a, const int it, PackShared<T> &sh, const int wl) {
    if (it >= a.nitems) {
        // no item: still take part in the launch chain
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        return;
    }
    const int4 item = a.items[it];
    if ((item.w & 15) == 0) {
        packed_body<T, 2, true>(a, item, sh, wl);
        return;
    }
    switch (item.z) {
        case 2: packed_body<T, 2, false>(a, item, sh, wl); break;
        case 3: packed_body<T, 3, false>(a, item, sh, wl); break;
        case 4: packed_body<T, 4, false>(a, item, sh, wl); break;
        case 5: packed_body<T, 5, false>(a, item, sh, wl); break;
        case 6: packed_body<T, 6, false>(a, item, sh, wl); break;
        case 7: packed_body<T, 7, false>(a, item, sh, wl); break;
        default: packed_body<T, 8, false>(a, item, sh, wl); break;
    }
}

template <typename T>
__global__ void __launch_bounds__(MOL_WARPS * 32, sizeof(T) == 4 ? MOL_MIN_BLOCKS : 1)
    molecule_packed_kernel(const MolArgs<T> a) {
    __shared__ PackShared<T> sh;
    const int wl = threadIdx.x >> 5;
    packed_item(a, (int)blockIdx.x * MOL_WARPS + wl, sh, wl);
}

template <typename T>
cudaError_t launch_molecules_packed(const MolArgs<T> &a, cudaStream_t s, bool pdl) {
    if (a.nitems == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.nitems + MOL_WARPS - 1) / MOL_WARPS);
    cfg.blockDim = dim3(MOL_WARPS * 32);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, molecule_packed_kernel<T>, a);
}

// Uniform-field form for two-level molecules: one thread per molecule, so that a warp
// streams 32 molecules' 2x2 matrices with 16-byte loads instead of one molecule's four
// elements.  The same step as molecule_body: E~ = gamma Eu (or the laser's wave) held
// over dt; the exact 2x2 exponential (kind 0) or nsub classic RK4 substeps of the GKSL
// equation (kind 1); mudot and the energy sum.  uniform_thread_step hands gamma <mu> of
// the new state to its caller: the cavity kernel sums it, the laser drive needs none.
template <typename T>
__device__ __forceinline__ void ld4(const cx<T> *p, cx<T> (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(p)), b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
        v[0] = {a.x, a.y}; v[1] = {a.z, a.w}; v[2] = {b.x, b.y}; v[3] = {b.z, b.w};
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + e);
            v[e] = {a.x, a.y};
        }
    }
}

template <typename T>
__device__ __forceinline__ void st4(cx<T> *p, const cx<T> (&v)[4]) {
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4 *>(p)[0] = make_float4(v[0].re, v[0].im, v[1].re, v[1].im);
        reinterpret_cast<float4 *>(p)[1] = make_float4(v[2].re, v[2].im, v[3].re, v[3].im);
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++) reinterpret_cast<double2 *>(p)[e] = make_double2(v[e].re, v[e].im);
    }
}

constexpr int MU_THREADS = MU_THREADS_HOST;


template <typename T, bool EXACT_ONLY>
__device__ __forceinline__ void uniform_thread_step(const MolArgs<T> &a, const int m, T (&gm)[3]) {
    const long long o = 4ll * m;
    const int kind = a.kind[m];
    const T gam = a.gamma[m];
    const double e_old = a.energy[m];
    // every load is independent of the others; a dipole component that is zero for the
    // whole ensemble is not read (one that is zero for some molecules is read as zeros)
    cx<T> r[4], h0[4], mu[3][4];
    ld4(a.rho + o, r);
    ld4(a.H0 + o, h0);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        if ((a.mu_zero >> c) & 1) {
#pragma unroll
            for (int e = 0; e < 4; e++) mu[c][e] = {T(0), T(0)};
        } else {
            ld4(a.mu + c * a.pool + o, mu[c]);
        }
    }
    T Et[3];
    uniform_field(a, m, Et);
#pragma unroll
    for (int c = 0; c < 3; c++) Et[c] *= gam;
    // H = H0 - Et . mu and <mu> before the step (Re Tr(rho A) = sum Re(rho_e conj(A_e)))
    cx<T> H[4];
    T mu0[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int e = 0; e < 4; e++) {
        H[e] = h0[e];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            H[e].re -= Et[c] * mu[c][e].re;
            H[e].im -= Et[c] * mu[c][e].im;
            mu0[c] += r[e].re * mu[c][e].re + r[e].im * mu[c][e].im;
        }
    }
    cx<T> r1[4];
    if (EXACT_ONLY || kind == 0) {
        const T dt = a.dt;
        const T z = T(0.5) * (H[0].re - H[3].re);
        const cx<T> b = H[1];
        const T W = sqrt(z * z + b.re * b.re + b.im * b.im);
        const T cw = cos(W * dt);
        const T sw = W > T(0) ? sin(W * dt) / W : dt;
        cx<T> U[4];
        U[0] = {cw, -sw * z};
        U[1] = {sw * b.im, -sw * b.re};
        U[2] = {-sw * b.im, -sw * b.re};
        U[3] = {cw, sw * z};
        cx<T> TT[4];
        for (int p = 0; p < 2; p++)
            for (int q = 0; q < 2; q++)
                TT[p * 2 + q] = cadd(cmul(U[p * 2 + 0], r[0 * 2 + q]), cmul(U[p * 2 + 1], r[1 * 2 + q]));
        for (int p = 0; p < 2; p++)
            for (int q = 0; q < 2; q++)
                r1[p * 2 + q] = cadd(cmul(TT[p * 2 + 0], cconj(U[q * 2 + 0])), cmul(TT[p * 2 + 1], cconj(U[q * 2 + 1])));
    } else if constexpr (!EXACT_ONLY) {
        const int ns = a.nsub[m];
        const T h = a.dt / T(ns);
        const T decay = a.decay[m], deph = a.dephase[m];
#pragma unroll
        for (int e = 0; e < 4; e++) r1[e] = r[e];
        for (int sstep = 0; sstep < ns; sstep++) {
            cx<T> base[4], S[4], acc[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                base[e] = r1[e];
                S[e] = r1[e];
                acc[e] = {T(0), T(0)};
            }
#pragma unroll
            for (int st = 0; st < 4; st++) {
                const T wgt = (st == 0 || st == 3) ? T(1) : T(2);
                const T cn = (st < 2) ? T(0.5) : T(1);
                cx<T> f[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    f[e] = rhs_elem(2, e >> 1, e & 1, S, H, decay, deph);
                    acc[e].re += wgt * f[e].re;
                    acc[e].im += wgt * f[e].im;
                }
                if (st < 3)
#pragma unroll
                    for (int e = 0; e < 4; e++) S[e] = {base[e].re + cn * h * f[e].re, base[e].im + cn * h * f[e].im};
            }
#pragma unroll
            for (int e = 0; e < 4; e++) {
                r1[e].re = base[e].re + h / T(6) * acc[e].re;
                r1[e].im = base[e].im + h / T(6) * acc[e].im;
            }
        }
    }
    st4(a.rho + o, r1);
    T mu1[3] = {T(0), T(0), T(0)};
    T en = T(0);
#pragma unroll
    for (int e = 0; e < 4; e++) {
#pragma unroll
        for (int c = 0; c < 3; c++) mu1[c] += r1[e].re * mu[c][e].re + r1[e].im * mu[c][e].im;
        en += r1[e].re * h0[e].re + r1[e].im * h0[e].im;
    }
    bool bad = false;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const T md = (mu1[c] - mu0[c]) / a.dt;
        a.Et[3 * m + c] = Et[c];
        a.mudot[3 * m + c] = md;
        gm[c] = gam * mu1[c];
        if (!isfinite(Et[c]) || !isfinite(md)) bad = true;
    }
    a.energy[m] = e_old + (double)en;
    if (bad) atomicCAS(a.status, 0, 6);
}

// Laser drive (no mode to feed).  EXACT_ONLY: every molecule takes the exact 2x2 step,
// so the RK4 branch (and its registers) is not compiled in, and four blocks of 256 fit
// on an SM.
template <typename T, bool EXACT_ONLY>
__global__ void __launch_bounds__(MU_THREADS, sizeof(T) == 4 ? (EXACT_ONLY ? MU_MIN_BLOCKS_EXACT : MU_MIN_BLOCKS) : 1)
    molecule_uniform_thread_kernel(const MolArgs<T> a) {
    const int m = blockIdx.x * MU_THREADS + threadIdx.x;
    T gm[3];
    if (m < a.nmol) uniform_thread_step<T, EXACT_ONLY>(a, m, gm);
}

// Single-mode cavity with two-level molecules, one launch per step: a fixed grid of at
// most CAV_GRID blocks walks the molecules (block b takes rows b, b + grid, ... of 256),
// each warp adds its 32 terms of gamma <mu> in the field type by the shuffle tree and
// accumulates its rows as an unevaluated pair hi + lo (Knuth's two-sum: FP32 operations
// that keep about twice the FP32 precision); the block writes the FP64 sum of its warps
// in warp order.  The block that takes the last ticket adds the partials in a fixed order
// (thread t: partials t, t + 256, ...; then a tree) and advances the mode.  No block
// waits for another; the grid, and so every sum, does not depend on the device.
template <typename T, bool EXACT_ONLY>
__global__ void __launch_bounds__(MU_THREADS, sizeof(T) == 4 ? MU_MIN_BLOCKS : 1)
    molecule_cavity_kernel(const MolArgs<T> a) {
    __shared__ double red[2][MU_THREADS];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    T hi[2] = {T(0), T(0)}, lo[2] = {T(0), T(0)};
    for (long long row = blockIdx.x; row * MU_THREADS < a.nmol; row += gridDim.x) {
        const long long m = row * MU_THREADS + tid;
        T gm[3] = {T(0), T(0), T(0)};
        if (m < a.nmol) uniform_thread_step<T, EXACT_ONLY>(a, (int)m, gm);
#pragma unroll
        for (int c = 0; c < 2; c++) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) gm[c] += __shfl_down_sync(0xffffffffu, gm[c], off);
            const T t = gm[c], sm = hi[c] + t, v = sm - hi[c];  // lane 0's t is the warp's sum
            lo[c] += (hi[c] - (sm - v)) + (t - v);
            hi[c] = sm;
        }
    }
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 2; c++) red[c][wp] = (double)hi[c] + (double)lo[c];
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int c = 0; c < 2; c++) {
            double sum = 0.0;
            for (int w = 0; w < MU_THREADS / 32; w++) sum += red[c][w];
            a.dpart[2 * blockIdx.x + c] = sum;
        }
        __threadfence();  // the partial is visible before the ticket is taken
        last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int c = 0; c < 2; c++) {
        double sum = 0.0;
        for (int b = tid; b < (int)gridDim.x; b += MU_THREADS) sum += __ldcg(a.dpart + 2 * b + c);
        red[c][tid] = sum;
    }
    __syncthreads();
    for (int o = MU_THREADS / 2; o > 0; o >>= 1) {
        if (tid < o)
#pragma unroll
            for (int c = 0; c < 2; c++) red[c][tid] += red[c][tid + o];
        __syncthreads();
    }
    if (tid != 0) return;
    const double d[2] = {red[0][0], red[1][0]};
    cavity_advance_mode(a.mode, a.euf, d, a.wc, a.eps, a.mdt);
    *a.ticket = 0u;  // ready for the next launch
}

// Uniform-field form (single-mode cavity): no window, no field read.
template <typename T, bool N2>
__global__ void __launch_bounds__(MOL_WARPS * 32, sizeof(T) == 4 ? MOL_MIN_BLOCKS : 1)
    molecule_uniform_kernel(const MolArgs<T> a) {
    molecule_body<T, SRC_UNIFORM, N2>(a, (int)blockIdx.x * MOL_WARPS);
}

// Batched form: one block per (instance, first molecule) work item, or, for an instance
// whose molecules take the packed form when it is stepped alone, per (instance, first
// packed item): the same arithmetic as that instance's own step.
template <typename T, bool N2>
__global__ void __launch_bounds__(MOL_WARPS * 32) molecule_batch_kernel(const MolBatch<T> b) {
    const int2 wk = b.work[blockIdx.x];
    const MolArgs<T> &a = b.args[2 * wk.x + ((b.lev0[wk.x] + b.s) & 1)];
    if (a.nitems > 0) {
        __shared__ PackShared<T> sh;
        const int wl = threadIdx.x >> 5;
        packed_item(a, wk.y + wl, sh, wl);
        return;
    }
    molecule_body<T, SRC_WINDOW, N2>(a, wk.y);
}

template <typename T>
cudaError_t launch_molecules_batch(const MolBatch<T> &b, int nwork, cudaStream_t s) {
    if (nwork == 0) return cudaSuccess;
    if (b.two_level)
        molecule_batch_kernel<T, true><<<nwork, MOL_WARPS * 32, 0, s>>>(b);
    else
        molecule_batch_kernel<T, false><<<nwork, MOL_WARPS * 32, 0, s>>>(b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_molecules_uniform(const MolArgs<T> &a, cudaStream_t s) {
    if (a.nmol == 0) return cudaSuccess;
    if (a.two_level) {
        if (a.dpart) return cudaErrorInvalidValue;  // a two-level cavity steps through launch_molecules_cavity
        const int nb = (a.nmol + MU_THREADS - 1) / MU_THREADS;
        if (a.exact_only)
            molecule_uniform_thread_kernel<T, true><<<nb, MU_THREADS, 0, s>>>(a);
        else
            molecule_uniform_thread_kernel<T, false><<<nb, MU_THREADS, 0, s>>>(a);
    } else {
        const int blocks = (a.nmol + MOL_WARPS - 1) / MOL_WARPS;
        molecule_uniform_kernel<T, false><<<blocks, MOL_WARPS * 32, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_molecules_cavity(const MolArgs<T> &a, cudaStream_t s) {
    if (a.nmol == 0 || !a.two_level || !a.dpart || !a.mode || !a.ticket) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(CAV_GRID, ((long long)a.nmol + MU_THREADS - 1) / MU_THREADS);
    if (a.exact_only)
        molecule_cavity_kernel<T, true><<<grid, MU_THREADS, 0, s>>>(a);
    else
        molecule_cavity_kernel<T, false><<<grid, MU_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_molecules(const MolArgs<T> &a, cudaStream_t s, bool pdl) {
    if (a.nmol == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((a.nmol + MOL_WARPS - 1) / MOL_WARPS);
    cfg.blockDim = dim3(MOL_WARPS * 32);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return a.two_level ? cudaLaunchKernelEx(&cfg, molecule_kernel<T, true>, a)
                     : cudaLaunchKernelEx(&cfg, molecule_kernel<T, false>, a);
}

// K3: weights.  One thread per (molecule, axis, stagger).  The raw window has
// wraw = 2R+2 entries starting at the (unwrapped) index s = floor(pos) - R; the
// entries are normalised to sum 1 and, on a periodic axis, folded onto the
// Wf = min(wraw, n) cells starting at the canonical start win.
template <typename T>
__global__ void weights_kernel(int nmol, const double *pos, const double *sigma, const int *win, const int *wf,
                               const int *wraw, int nx, int ny, int nz, int p0, int p1, int p2, T *w) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nmol * 6) return;
    const int m = t / 6, ax = (t % 6) / 2, st = t % 2;
    const int n = ax == 0 ? nx : (ax == 1 ? ny : nz);
    const int per = ax == 0 ? p0 : (ax == 1 ? p1 : p2);
    const double p = pos[3 * m + ax], sg = sigma[m];
    const int W = wraw[3 * m + ax];
    const int R = (W - 2) / 2;
    const int s = (int)floor(p) - R;
    double v[32];
    double sum = 0.0;
    // exponent relative to the nearest sample (the largest weight is 1): the normalisation
    // removes the common factor, and a narrow kernel cannot underflow to 0/0
    const double fc = p - 0.5 * st, dn = fc - floor(fc + 0.5);
    for (int q = 0; q < W; q++) {
        double x = (double)(s + q) + 0.5 * st - p;
        v[q] = exp(-(x * x - dn * dn) / (2.0 * sg * sg));
        sum += v[q];
    }
    double f[WMAX];
    for (int q = 0; q < WMAX; q++) f[q] = 0.0;
    const int Wf = (wf[m] >> (8 * ax)) & 0xff;
    const int start = win[3 * m + ax];
    for (int q = 0; q < W; q++) {
        int c = s + q;
        int d;
        if (per) {
            int cc = ((c % n) + n) % n;
            d = cc - start;
            if (d < 0) d += n;
        } else {
            d = c - start;
        }
        if (d >= 0 && d < Wf) f[d] += v[q] / sum;
    }
    T *out = w + (long long)m * NW + (2 * ax + st) * WMAX;
    for (int q = 0; q < WMAX; q++) out[q] = (T)f[q];
}

template <typename T>
cudaError_t launch_weights(int nmol, const double *pos, const double *sigma, const int *win, const int *wf,
                           const int *wraw, const int *dims, const int *per, T *w, cudaStream_t s) {
    if (nmol == 0) return cudaSuccess;
    int threads = 128, blocks = (nmol * 6 + threads - 1) / threads;
    weights_kernel<T><<<blocks, threads, 0, s>>>(nmol, pos, sigma, win, wf, wraw, dims[0], dims[1], dims[2], per[0],
                                                  per[1], per[2], w);
    return cudaGetLastError();
}

template <typename T>
__global__ void mol_export_kernel(int what, int nmol, const int *nlev, const long long *off, const cx<T> *rho,
                                  const T *Et, const T *mudot, const double *energy, long long pool, double *dst) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (what == 0) {
        if (t < pool) { dst[2 * t] = (double)rho[t].re; dst[2 * t + 1] = (double)rho[t].im; }
    } else if (what == 1 || what == 2) {
        if (t < 3ll * nmol) dst[t] = (double)(what == 1 ? Et[t] : mudot[t]);
    } else if (what == 3) {
        if (t < nmol) dst[t] = energy[t];
    } else if (what == 4) {
        if (t < (long long)nmol * MAXLEV) {
            int m = (int)(t / MAXLEV), l = (int)(t % MAXLEV);
            int n = nlev[m];
            dst[t] = l < n ? (double)rho[off[m] + l * n + l].re : 0.0;
        }
    }
}

template <typename T>
cudaError_t launch_mol_export(int what, int nmol, const int *nlev, const long long *off, const cx<T> *rho,
                              const T *Et, const T *mudot, const double *energy, long long pool, double *dst,
                              cudaStream_t s) {
    long long n = what == 0 ? pool : (what == 3 ? nmol : (what == 4 ? (long long)nmol * MAXLEV : 3ll * nmol));
    if (n == 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    mol_export_kernel<T><<<blocks, 256, 0, s>>>(what, nmol, nlev, off, rho, Et, mudot, energy, pool, dst);
    return cudaGetLastError();
}

#define ML_INST(T)                                                                                              \
    template cudaError_t launch_molecules<T>(const MolArgs<T> &, cudaStream_t, bool);                           \
    template cudaError_t launch_molecules_packed<T>(const MolArgs<T> &, cudaStream_t, bool);                    \
    template cudaError_t launch_molecules_uniform<T>(const MolArgs<T> &, cudaStream_t);                         \
    template cudaError_t launch_molecules_cavity<T>(const MolArgs<T> &, cudaStream_t);                          \
    template cudaError_t launch_molecules_batch<T>(const MolBatch<T> &, int, cudaStream_t);                     \
    template cudaError_t launch_weights<T>(int, const double *, const double *, const int *, const int *,       \
                                           const int *, const int *, const int *, T *, cudaStream_t);           \
    template cudaError_t launch_mol_export<T>(int, int, const int *, const long long *, const cx<T> *, const T *, \
                                              const T *, const double *, long long, double *, cudaStream_t);
ML_INST(float)
ML_INST(double)

}  // namespace ml
