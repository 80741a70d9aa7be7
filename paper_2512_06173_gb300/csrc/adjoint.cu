// Discrete adjoint of the coupled step: gradients of a DFT flux (the Sec. IV
// spectra) with respect to the permittivity of every design-box cell and the
// coupling gamma_m of every molecule, with checkpoint-and-recompute of the field
// history.
//
// Adjoint variables, in the padded layout of the fields:
//   U    = Ebar / eps  (adjoint of E divided by the cell's relative permittivity),
//   Hbar               (adjoint of H),
// and, per CPML slab and layer pair, one adjoint memory for each convolution of
// the E update (phi) and of the H update (chi).  For a convolution that enters a
// curl component with sign s, the forward pair  psi' = b psi + c d,  term = s (kinv d
// + psi')  has the transpose  w = kinv u + c (m + u),  dbar = s w,  m' = b (m + u),
// with u the adjoint of the curl component and m the memory (kept multiplied by s,
// so that every pair uses the same update).  Outside a layer w = u.
//
// Reversing the step that took E^n to E^{n+1} keeps the forward launch order:
//   gather of U^{n+1} over the molecule windows (the forward gather kernel),
//   molecule kernel: adjoint of rho and of the regularised field (Eq. E_regu_Emi,
//     Eq. von-Neumann-tls, Eq. dipole_derivative reversed),
//   current kernel with amplitudes -gamma Etbar / dt (the forward kernel),
//   pass A: Hbar^{n+1/2} += transpose of the E update applied to u = dt U^{n+1},
//           + d objective / d H^{n+1/2}; permittivity gradient,
//   pass B: U^n = U^{n+1} + (dt/eps)/dt (transpose of the H update applied to
//           v = -dt Hbar, Drude, d objective / d E^n) - (dt/eps) J,
// with tangential U on the index-0 PEC walls held at zero.
#include <algorithm>
#include <cmath>
#include <vector>

#include "grid.cuh"

namespace ml {

template <typename T>
struct AdjFieldArgs {
    int nx, ny, nz, px;
    long long plane;
    int per[3], pml[6];
    T dt;
    T *U[3];
    T *Hb[3];
    const T *cpml[3];
    const T *phi_in[3][2];
    T *phi_out[3][2];
    const T *chi_in[3][2];
    T *chi_out[3][2];
    const uint8_t *mat;
    const T *mat_cb, *mat_dk, *mat_db, *mat_dp;
    int dbox[6];
    const T *dcb;
    int jbox[6];
    int npole;               // pole slots in use
    long long jcnt;          // cells of the pole box
    T *JDb;                  // adjoint of each slot's pole current, [slot][component][jcnt] (null: no poles)
    T *PDb;                  // adjoint of each slot's polarisation, same layout (null: no Lorentz pole)
    int jb0[3], jbn[3];
    const T *Jb[3];
    T *gseg;                 // design-box gradient of the current segment (pass A), or null
    const T *Eprev, *Enext;  // design-box E^n and E^{n+1} (3 x nbox each)
    long long nbox;
    int pax, pidx, pnb;      // objective plane: axis, index, cells along b
    int pim, hasm;           // index of the layer below the plane (wrapped), and whether it exists
    // d objective / d (E_b, E_c, H_b, H_c) at plane cell o for a sample at time t is
    // cos(w t) tab[q][o].re + sin(w t) tab[q][o].im (table built once per run)
    const cx<T> *tab;        // 4 x ncell, or null
    T csH, snH, csE, snE;    // cos, sin of w t for the H sample (pass A) and E sample (pass B)
    int injectE;
};

__device__ __forceinline__ int adj_slab(int p, int n, int lo, int hi) {
    if (p < lo) return p;
    if (p >= n - hi) return p - (n - hi) + lo;
    return -1;
}

template <typename T>
__device__ __forceinline__ long long adj_gidx(const AdjFieldArgs<T> &a, int i, int j, int k) {
    return (long long)(k + 1) * a.plane + (long long)(j + 1) * a.px + (i + XO);
}

// index of cell (i,j,k) in the slab storage of axis ax (slab coordinate s)
template <typename T>
__device__ __forceinline__ long long adj_midx(const AdjFieldArgs<T> &a, int ax, int s, int i, int j, int k) {
    if (ax == 0) return ((long long)k * a.ny + j) * (a.pml[0] + a.pml[1]) + s;
    if (ax == 1) return ((long long)k * (a.pml[2] + a.pml[3]) + s) * a.nx + i;
    return ((long long)s * a.ny + j) * a.nx + i;
}

// Weighted adjoint of one curl term at cell (i,j,k) whose derivative runs along ax
// (pair q of that axis).  side 0: E-update terms (bE cE kE, memory phi); side 1:
// H-update terms (bH cH kH, memory chi).
template <typename T>
__device__ __forceinline__ T wterm(const AdjFieldArgs<T> &a, int side, int ax, int q, int i, int j, int k, T u) {
    const int p = ax == 0 ? i : (ax == 1 ? j : k);
    const int n = ax == 0 ? a.nx : (ax == 1 ? a.ny : a.nz);
    const int s = adj_slab(p, n, a.pml[2 * ax], a.pml[2 * ax + 1]);
    if (s < 0) return u;
    const T *cf = a.cpml[ax];
    const T c = cf[(side * 3 + 1) * n + p], kinv = cf[(side * 3 + 2) * n + p];
    const long long m = adj_midx(a, ax, s, i, j, k);
    const T mem = side == 0 ? a.phi_in[ax][q][m] : a.chi_in[ax][q][m];
    return kinv * u + c * (mem + u);
}

template <typename T>
__device__ __forceinline__ void mstore(const AdjFieldArgs<T> &a, int side, int ax, int q, int i, int j, int k, T u) {
    const int p = ax == 0 ? i : (ax == 1 ? j : k);
    const int n = ax == 0 ? a.nx : (ax == 1 ? a.ny : a.nz);
    const int s = adj_slab(p, n, a.pml[2 * ax], a.pml[2 * ax + 1]);
    if (s < 0) return;
    const T b = a.cpml[ax][(side * 3) * n + p];
    const long long m = adj_midx(a, ax, s, i, j, k);
    if (side == 0) a.phi_out[ax][q][m] = b * (a.phi_in[ax][q][m] + u);
    else a.chi_out[ax][q][m] = b * (a.chi_in[ax][q][m] + u);
}

// dt/eps of the cell and its material index
template <typename T>
__device__ __forceinline__ T adj_cb(const AdjFieldArgs<T> &a, int i, int j, int k, int &midx) {
    midx = a.mat ? a.mat[((long long)k * a.ny + j) * a.nx + i] : 0;
    T cb = a.mat_cb[midx];
    if (a.dcb && i >= a.dbox[0] && i < a.dbox[0] + a.dbox[3] && j >= a.dbox[1] && j < a.dbox[1] + a.dbox[4] &&
        k >= a.dbox[2] && k < a.dbox[2] + a.dbox[5])
        cb = a.dcb[((long long)(k - a.dbox[2]) * a.dbox[4] + (j - a.dbox[1])) * a.dbox[3] + (i - a.dbox[0])];
    return cb;
}

// components held at zero by an index-0 PEC wall (bit c)
template <typename T>
__device__ __forceinline__ int adj_forced(const AdjFieldArgs<T> &a, int i, int j, int k) {
    const bool wx = !a.per[0] && i == 0, wy = !a.per[1] && j == 0, wz = !a.per[2] && k == 0;
    return ((wy || wz) ? 1 : 0) | ((wx || wz) ? 2 : 0) | ((wx || wy) ? 4 : 0);
}

// cos(w t) re + sin(w t) im of one table entry
template <typename T>
__device__ __forceinline__ T adj_phase(cx<T> e, T cs, T sn) { return cs * e.re + sn * e.im; }

constexpr int AZC = 8;  // z planes per thread column in the adjoint passes

// CPML coefficients (b, c, kinv) of one side (0: E update, 1: H update) at index p of axis ax
template <typename T>
__device__ __forceinline__ void adj_coef(const AdjFieldArgs<T> &a, int side, int ax, int n, int p, T &b, T &c, T &k) {
    const T *cf = a.cpml[ax];
    b = cf[(side * 3) * n + p];
    c = cf[(side * 3 + 1) * n + p];
    k = cf[(side * 3 + 2) * n + p];
}

// Pass A: Hbar^{n+1/2} += transpose of the E update applied to u = dt U^{n+1} (with the
// E-side CPML memories phi), + d objective / d H^{n+1/2}; d objective / d eps.  One
// thread per (x, y) column marching AZC planes up in z; U of the column's next plane
// is carried to the following iteration.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) adj_passA_kernel(const AdjFieldArgs<T> a) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * AZC, k1 = min(k0 + AZC, a.nz);
    if (i >= a.nx || j >= a.ny) return;
    const T dt = a.dt;
    int xp = i + 1, yp = j + 1;
    bool vx = true, vy = true;
    if (xp == a.nx) { if (a.per[0]) xp = 0; else vx = false; }
    if (yp == a.ny) { if (a.per[1]) yp = 0; else vy = false; }
    const int dxt = a.pml[0] + a.pml[1], dyt = a.pml[2] + a.pml[3];
    const int sx = adj_slab(i, a.nx, a.pml[0], a.pml[1]), sxp = vx ? adj_slab(xp, a.nx, a.pml[0], a.pml[1]) : -1;
    const int sy = adj_slab(j, a.ny, a.pml[2], a.pml[3]), syp = vy ? adj_slab(yp, a.ny, a.pml[2], a.pml[3]) : -1;
    T bx = 0, cx = 0, kx = 1, bxp = 0, cxp = 0, kxp = 1, by = 0, cy = 0, ky = 1, byp = 0, cyp = 0, kyp = 1;
    if (sx >= 0) adj_coef(a, 0, 0, a.nx, i, bx, cx, kx);
    if (sxp >= 0) adj_coef(a, 0, 0, a.nx, xp, bxp, cxp, kxp);
    if (sy >= 0) adj_coef(a, 0, 1, a.ny, j, by, cy, ky);
    if (syp >= 0) adj_coef(a, 0, 1, a.ny, yp, byp, cyp, kyp);
    const long long ro = (long long)(j + 1) * a.px + i + XO;
    const long long rx = (long long)(j + 1) * a.px + xp + XO;
    const long long ry = (long long)(yp + 1) * a.px + i + XO;
    const T *U0 = a.U[0], *U1 = a.U[1], *U2 = a.U[2];
    const bool inbx = a.gseg && i >= a.dbox[0] && i < a.dbox[0] + a.dbox[3] && j >= a.dbox[1] && j < a.dbox[1] + a.dbox[4];
    long long pk = (long long)(k0 + 1) * a.plane;
    T c0 = U0[pk + ro], c1 = U1[pk + ro], c2 = U2[pk + ro];
    for (int k = k0; k < k1; k++, pk += a.plane) {
        int zp = k + 1;
        bool vz = true;
        if (zp == a.nz) { if (a.per[2]) zp = 0; else vz = false; }
        T n0 = T(0), n1 = T(0), n2 = T(0);
        if (vz) {
            const long long pz = (long long)(zp + 1) * a.plane + ro;
            n0 = U0[pz];
            n1 = U1[pz];
            n2 = U2[pz];
        }
        T w1xp = T(0), w2xp = T(0), w0yp = T(0), w2yp = T(0);
        if (vx) { w1xp = dt * U1[pk + rx]; w2xp = dt * U2[pk + rx]; }
        if (vy) { w0yp = dt * U0[pk + ry]; w2yp = dt * U2[pk + ry]; }
        const T u0 = dt * c0, u1 = dt * c1, u2 = dt * c2;
        T w1x = u1, w2x = u2, w0y = u0, w2y = u2, w0z = u0, w1z = u1;
        T w0zp = dt * n0, w1zp = dt * n1;
        // CPML: pairs x (comp 1, comp 2), y (comp 0, comp 2), z (comp 0, comp 1)
        if (sx >= 0) {
            const long long q = ((long long)k * a.ny + j) * dxt + sx;
            const T p0 = a.phi_in[0][0][q], p1 = a.phi_in[0][1][q];
            w1x = kx * u1 + cx * (p0 + u1);
            w2x = kx * u2 + cx * (p1 + u2);
            a.phi_out[0][0][q] = bx * (p0 + u1);
            a.phi_out[0][1][q] = bx * (p1 + u2);
        }
        if (sxp >= 0) {
            const long long q = ((long long)k * a.ny + j) * dxt + sxp;
            w1xp = kxp * w1xp + cxp * (a.phi_in[0][0][q] + w1xp);
            w2xp = kxp * w2xp + cxp * (a.phi_in[0][1][q] + w2xp);
        }
        if (sy >= 0) {
            const long long q = ((long long)k * dyt + sy) * a.nx + i;
            const T p0 = a.phi_in[1][0][q], p1 = a.phi_in[1][1][q];
            w0y = ky * u0 + cy * (p0 + u0);
            w2y = ky * u2 + cy * (p1 + u2);
            a.phi_out[1][0][q] = by * (p0 + u0);
            a.phi_out[1][1][q] = by * (p1 + u2);
        }
        if (syp >= 0) {
            const long long q = ((long long)k * dyt + syp) * a.nx + i;
            w0yp = kyp * w0yp + cyp * (a.phi_in[1][0][q] + w0yp);
            w2yp = kyp * w2yp + cyp * (a.phi_in[1][1][q] + w2yp);
        }
        if (a.pml[4] | a.pml[5]) {
            const int sz = adj_slab(k, a.nz, a.pml[4], a.pml[5]);
            if (sz >= 0) {
                T bz, cz, kz;
                adj_coef(a, 0, 2, a.nz, k, bz, cz, kz);
                const long long q = ((long long)sz * a.ny + j) * a.nx + i;
                const T p0 = a.phi_in[2][0][q], p1 = a.phi_in[2][1][q];
                w0z = kz * u0 + cz * (p0 + u0);
                w1z = kz * u1 + cz * (p1 + u1);
                a.phi_out[2][0][q] = bz * (p0 + u0);
                a.phi_out[2][1][q] = bz * (p1 + u1);
            }
            const int szp = vz ? adj_slab(zp, a.nz, a.pml[4], a.pml[5]) : -1;
            if (szp >= 0) {
                T bz, cz, kz;
                adj_coef(a, 0, 2, a.nz, zp, bz, cz, kz);
                const long long q = ((long long)szp * a.ny + j) * a.nx + i;
                w0zp = kz * w0zp + cz * (a.phi_in[2][0][q] + w0zp);
                w1zp = kz * w1zp + cz * (a.phi_in[2][1][q] + w1zp);
            }
        }
        // E update: curl0 = dHz/dy - dHy/dz, curl1 = dHx/dz - dHz/dx, curl2 = dHy/dx - dHx/dy
        // with backward differences of H; their transposes are forward differences.
        const long long g = pk + ro;
        T hx = a.Hb[0][g] + (w1z - w1zp) - (w2y - w2yp);
        T hy = a.Hb[1][g] + (w2x - w2xp) - (w0z - w0zp);
        T hz = a.Hb[2][g] + (w0y - w0yp) - (w1x - w1xp);
        // d objective / d H^{n+1/2}: the plane's H sums take the mean of the cells at the
        // plane index and the one below it
        if (a.tab) {
            const int pc = a.pax == 0 ? i : (a.pax == 1 ? j : k);
            const int mult = (pc == a.pidx ? 1 : 0) + ((a.hasm && pc == a.pim) ? 1 : 0);
            if (mult) {
                const int u = a.pax == 0 ? j : (a.pax == 1 ? k : i);
                const int v = a.pax == 0 ? k : (a.pax == 1 ? i : j);
                const long long o = (long long)v * a.pnb + u;
                const long long nc = (long long)a.pnb * (a.pax == 0 ? a.nz : (a.pax == 1 ? a.nx : a.ny));
                const T db = T(mult) * adj_phase(a.tab[2 * nc + o], a.csH, a.snH);
                const T dc = T(mult) * adj_phase(a.tab[3 * nc + o], a.csH, a.snH);
                if (a.pax == 0) { hy += db; hz += dc; }
                else if (a.pax == 1) { hz += db; hx += dc; }
                else { hx += db; hy += dc; }
            }
        }
        a.Hb[0][g] = hx;
        a.Hb[1][g] = hy;
        a.Hb[2][g] = hz;
        // d/d eps of E^{n+1} = E^n + dt/eps (...) is -(E^{n+1} - E^n)/eps; with U = Ebar/eps
        if (inbx && k >= a.dbox[2] && k < a.dbox[2] + a.dbox[5]) {
            const long long q = ((long long)(k - a.dbox[2]) * a.dbox[4] + (j - a.dbox[1])) * a.dbox[3] + (i - a.dbox[0]);
            a.gseg[q] -= c0 * (a.Enext[q] - a.Eprev[q]) + c1 * (a.Enext[a.nbox + q] - a.Eprev[a.nbox + q]) +
                         c2 * (a.Enext[2 * a.nbox + q] - a.Eprev[2 * a.nbox + q]);
        }
        c0 = n0;
        c1 = n1;
        c2 = n2;
    }
}

// Pass B: U^n = U^{n+1} + (1/eps)(transpose of the H update applied to v = -dt Hbar,
// with the H-side memories chi; Drude; d objective / d E^n) - (dt/eps) J, tangential
// U on index-0 walls held at 0.  Column march as in pass A; the z-pair terms of the
// plane below are carried.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) adj_passB_kernel(const AdjFieldArgs<T> a) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
    const int k0 = blockIdx.z * AZC, k1 = min(k0 + AZC, a.nz);
    if (i >= a.nx || j >= a.ny) return;
    const T dt = a.dt;
    int xm = i - 1, ym = j - 1;
    bool vx = true, vy = true;
    if (xm < 0) { if (a.per[0]) xm = a.nx - 1; else vx = false; }
    if (ym < 0) { if (a.per[1]) ym = a.ny - 1; else vy = false; }
    const int dxt = a.pml[0] + a.pml[1], dyt = a.pml[2] + a.pml[3];
    const int sx = adj_slab(i, a.nx, a.pml[0], a.pml[1]), sxm = vx ? adj_slab(xm, a.nx, a.pml[0], a.pml[1]) : -1;
    const int sy = adj_slab(j, a.ny, a.pml[2], a.pml[3]), sym = vy ? adj_slab(ym, a.ny, a.pml[2], a.pml[3]) : -1;
    T bx = 0, cx = 0, kx = 1, bxm = 0, cxm = 0, kxm = 1, by = 0, cy = 0, ky = 1, bym = 0, cym = 0, kym = 1;
    if (sx >= 0) adj_coef(a, 1, 0, a.nx, i, bx, cx, kx);
    if (sxm >= 0) adj_coef(a, 1, 0, a.nx, xm, bxm, cxm, kxm);
    if (sy >= 0) adj_coef(a, 1, 1, a.ny, j, by, cy, ky);
    if (sym >= 0) adj_coef(a, 1, 1, a.ny, ym, bym, cym, kym);
    const long long ro = (long long)(j + 1) * a.px + i + XO;
    const long long rx = (long long)(j + 1) * a.px + xm + XO;
    const long long ry = (long long)(ym + 1) * a.px + i + XO;
    const T *H0 = a.Hb[0], *H1 = a.Hb[1], *H2 = a.Hb[2];
    const bool zl = (a.pml[4] | a.pml[5]) != 0;
    // z-pair terms (comp 0, comp 1) of the cell below the first plane
    T w0zm = T(0), w1zm = T(0);
    {
        int zm = k0 - 1;
        bool vz = true;
        if (zm < 0) { if (a.per[2]) zm = a.nz - 1; else vz = false; }
        if (vz) {
            const long long q = (long long)(zm + 1) * a.plane + ro;
            w0zm = -dt * H0[q];
            w1zm = -dt * H1[q];
            const int szm = zl ? adj_slab(zm, a.nz, a.pml[4], a.pml[5]) : -1;
            if (szm >= 0) {
                T bz, cz, kz;
                adj_coef(a, 1, 2, a.nz, zm, bz, cz, kz);
                const long long m = ((long long)szm * a.ny + j) * a.nx + i;
                w0zm = kz * w0zm + cz * (a.chi_in[2][0][m] + w0zm);
                w1zm = kz * w1zm + cz * (a.chi_in[2][1][m] + w1zm);
            }
        }
    }
    const int forced_xy = (!a.per[0] && i == 0 ? 1 : 0) | (!a.per[1] && j == 0 ? 2 : 0);
    long long pk = (long long)(k0 + 1) * a.plane;
    for (int k = k0; k < k1; k++, pk += a.plane) {
        const long long g = pk + ro;
        const T v0 = -dt * H0[g], v1 = -dt * H1[g], v2 = -dt * H2[g];
        T w1xm = T(0), w2xm = T(0), w0ym = T(0), w2ym = T(0);
        if (vx) { w1xm = -dt * H1[pk + rx]; w2xm = -dt * H2[pk + rx]; }
        if (vy) { w0ym = -dt * H0[pk + ry]; w2ym = -dt * H2[pk + ry]; }
        T w1x = v1, w2x = v2, w0y = v0, w2y = v2, w0z = v0, w1z = v1;
        if (sx >= 0) {
            const long long q = ((long long)k * a.ny + j) * dxt + sx;
            const T p0 = a.chi_in[0][0][q], p1 = a.chi_in[0][1][q];
            w1x = kx * v1 + cx * (p0 + v1);
            w2x = kx * v2 + cx * (p1 + v2);
            a.chi_out[0][0][q] = bx * (p0 + v1);
            a.chi_out[0][1][q] = bx * (p1 + v2);
        }
        if (sxm >= 0) {
            const long long q = ((long long)k * a.ny + j) * dxt + sxm;
            w1xm = kxm * w1xm + cxm * (a.chi_in[0][0][q] + w1xm);
            w2xm = kxm * w2xm + cxm * (a.chi_in[0][1][q] + w2xm);
        }
        if (sy >= 0) {
            const long long q = ((long long)k * dyt + sy) * a.nx + i;
            const T p0 = a.chi_in[1][0][q], p1 = a.chi_in[1][1][q];
            w0y = ky * v0 + cy * (p0 + v0);
            w2y = ky * v2 + cy * (p1 + v2);
            a.chi_out[1][0][q] = by * (p0 + v0);
            a.chi_out[1][1][q] = by * (p1 + v2);
        }
        if (sym >= 0) {
            const long long q = ((long long)k * dyt + sym) * a.nx + i;
            w0ym = kym * w0ym + cym * (a.chi_in[1][0][q] + w0ym);
            w2ym = kym * w2ym + cym * (a.chi_in[1][1][q] + w2ym);
        }
        if (zl) {
            const int sz = adj_slab(k, a.nz, a.pml[4], a.pml[5]);
            if (sz >= 0) {
                T bz, cz, kz;
                adj_coef(a, 1, 2, a.nz, k, bz, cz, kz);
                const long long q = ((long long)sz * a.ny + j) * a.nx + i;
                const T p0 = a.chi_in[2][0][q], p1 = a.chi_in[2][1][q];
                w0z = kz * v0 + cz * (p0 + v0);
                w1z = kz * v1 + cz * (p1 + v1);
                a.chi_out[2][0][q] = bz * (p0 + v0);
                a.chi_out[2][1][q] = bz * (p1 + v1);
            }
        }
        // H update: cx = dEz/dy - dEy/dz, cy = dEx/dz - dEz/dx, cz = dEy/dx - dEx/dy with
        // forward differences of E; their transposes are backward differences.
        T d0 = (w1zm - w1z) - (w2ym - w2y);
        T d1 = (w0z - w0zm) + (w2xm - w2x);
        T d2 = (w0ym - w0y) - (w1xm - w1x);
        w0zm = w0z;
        w1zm = w1z;
        const T o0 = a.U[0][g], o1 = a.U[1][g], o2 = a.U[2][g];
        int midx;
        const T cb = adj_cb(a, i, j, k, midx);
        // dispersive poles, slot by slot: J' = dk J + db E^n - dp P, used in the E update as
        // -dt/eps J'; Lorentz (dp != 0): P' = P + dt J'.  The adjoint of J' collects the E
        // update's -dt U, the carried adjoint of J' and, through P', dt Pbar'.
        if (a.JDb && i >= a.jbox[0] && i < a.jbox[0] + a.jbox[3] && j >= a.jbox[1] && j < a.jbox[1] + a.jbox[4] &&
            k >= a.jbox[2] && k < a.jbox[2] + a.jbox[5]) {
            const long long jq = ((long long)(k - a.jbox[2]) * a.jbox[4] + (j - a.jbox[1])) * a.jbox[3] + (i - a.jbox[0]);
            const long long jc = a.jcnt;
            for (int p = 0; p < a.npole; p++) {
                const int mk = midx * ML_MAX_POLES + p;
                const T db = a.mat_db[mk];
                if (db == T(0)) break;  // a material's poles fill slots 0, 1, ...
                const T dk = a.mat_dk[mk];
                const T dp = a.PDb ? a.mat_dp[mk] : T(0);
                T *Jb = a.JDb + 3 * p * jc + jq;
                T t0 = Jb[0] - dt * o0, t1 = Jb[jc] - dt * o1, t2 = Jb[2 * jc] - dt * o2;
                if (dp != T(0)) {
                    T *Pb = a.PDb + 3 * p * jc + jq;
                    t0 += dt * Pb[0];
                    t1 += dt * Pb[jc];
                    t2 += dt * Pb[2 * jc];
                    Pb[0] -= dp * t0;
                    Pb[jc] -= dp * t1;
                    Pb[2 * jc] -= dp * t2;
                }
                Jb[0] = dk * t0;
                Jb[jc] = dk * t1;
                Jb[2 * jc] = dk * t2;
                d0 += db * t0;
                d1 += db * t1;
                d2 += db * t2;
            }
        }
        // d objective / d E^n (sampled by the step before this one)
        if (a.injectE && a.tab && (a.pax == 0 ? i : (a.pax == 1 ? j : k)) == a.pidx) {
            const int u = a.pax == 0 ? j : (a.pax == 1 ? k : i);
            const int v = a.pax == 0 ? k : (a.pax == 1 ? i : j);
            const long long o = (long long)v * a.pnb + u;
            const long long nc = (long long)a.pnb * (a.pax == 0 ? a.nz : (a.pax == 1 ? a.nx : a.ny));
            const T db = adj_phase(a.tab[o], a.csE, a.snE), dc = adj_phase(a.tab[nc + o], a.csE, a.snE);
            if (a.pax == 0) { d1 += db; d2 += dc; }
            else if (a.pax == 1) { d2 += db; d0 += dc; }
            else { d0 += db; d1 += dc; }
        }
        T J0 = T(0), J1 = T(0), J2 = T(0);
        if (a.Jb[0] || a.Jb[1] || a.Jb[2]) {
            const int xr = i - a.jb0[0], yr = j - a.jb0[1], kr = k - a.jb0[2];
            if ((unsigned)xr < (unsigned)a.jbn[0] && (unsigned)yr < (unsigned)a.jbn[1] &&
                (unsigned)kr < (unsigned)a.jbn[2]) {
                const long long q = ((long long)kr * a.jbn[1] + yr) * a.jbn[0] + xr;
                if (a.Jb[0]) J0 = a.Jb[0][q];
                if (a.Jb[1]) J1 = a.Jb[1][q];
                if (a.Jb[2]) J2 = a.Jb[2][q];
            }
        }
        const T inv = cb / dt;  // 1/eps
        const bool wz = !a.per[2] && k == 0;
        const bool f0 = (forced_xy & 2) || wz, f1 = (forced_xy & 1) || wz, f2 = forced_xy != 0;
        a.U[0][g] = f0 ? T(0) : o0 + inv * d0 - cb * J0;
        a.U[1][g] = f1 ? T(0) : o1 + inv * d1 - cb * J1;
        a.U[2][g] = f2 ? T(0) : o2 + inv * d2 - cb * J2;
    }
}

// d objective / d E^N of the last sample, added to U before the reverse sweep.
template <typename T>
__global__ void adj_inject_kernel(const AdjFieldArgs<T> a, int nc) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)a.pnb * nc) return;
    const int u = (int)(t % a.pnb), v = (int)(t / a.pnb);
    const int ax = a.pax, b = (ax + 1) % 3, c = (ax + 2) % 3;
    int pc[3];
    pc[ax] = a.pidx;
    pc[b] = u;
    pc[c] = v;
    const long long ncell = (long long)a.pnb * nc;
    const T db = adj_phase(a.tab[t], a.csE, a.snE), dc = adj_phase(a.tab[ncell + t], a.csE, a.snE);
    int midx;
    const T inv = adj_cb(a, pc[0], pc[1], pc[2], midx) / a.dt;
    const int forced = adj_forced(a, pc[0], pc[1], pc[2]);
    const long long g = adj_gidx(a, pc[0], pc[1], pc[2]);
    if (!((forced >> b) & 1)) a.U[b][g] += inv * db;
    if (!((forced >> c) & 1)) a.U[c][g] += inv * dc;
}

// Objective J = Re sum_o (E_b,o conj(H_c,o) - E_c,o conj(H_b,o)) with the sums
// E = sum_n e^{i w t_E} dt E^{n+1}, H = sum_n e^{i w t_H} dt (mean of H^{n+1/2} over the
// plane and the layer below).  Its derivative with respect to one sample is
// Re(e^{i w t} c) for a fixed complex c per cell and component:
//   E_b: dt conj(H_c)   E_c: -dt conj(H_b)   H_b (each of the two cells): -dt E_c / 2
//   H_c: dt E_b / 2,
// stored as (Re c, -Im c) so that Re(e^{i w t} c) = cos(w t) re + sin(w t) im.
template <typename T>
__global__ void adj_table_kernel(const double2 *acc, long long ncell, double dt, cx<T> *tab) {
    const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (o >= ncell) return;
    const double2 e1 = acc[o], e2 = acc[ncell + o], h1 = acc[2 * ncell + o], h2 = acc[3 * ncell + o];
    tab[o] = {(T)(dt * h2.x), (T)(dt * h2.y)};
    tab[ncell + o] = {(T)(-dt * h1.x), (T)(-dt * h1.y)};
    tab[2 * ncell + o] = {(T)(-0.5 * dt * e2.x), (T)(-0.5 * dt * e2.y)};
    tab[3 * ncell + o] = {(T)(0.5 * dt * e1.x), (T)(0.5 * dt * e1.y)};
}

// FP64 total of the design-box gradient += the segment's sum; the segment sum restarts.
template <typename T>
__global__ void adj_fold_kernel(T *gseg, double *geps, long long n) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= n) return;
    geps[q] += (double)gseg[q];
    gseg[q] = T(0);
}

template <typename T>
struct AdjMolArgs {
    int nmol;
    T dt;
    const int *kind;          // 0: exact two-level; 1: RK4 GKSL
    const int *nlev, *nsub;
    const T *decay, *dephase;
    const int *cmask;
    const long long *off;
    const T *gamma;
    const cx<T> *H0, *mu;
    long long pool;
    const int *moff, *mlist;
    const T *part;
    const cx<T> *rho_n;       // rho^n (pool)
    const T *Et_n, *md_n;     // field and mudot of the forward step (3 per molecule)
    cx<T> *rhob;              // adjoint of rho (pool): rho^{n+1} in, rho^n out
    T *cadj;                  // current amplitudes for the adjoint scatter
    double *ggam;             // d objective / d gamma (accumulated)
};

template <typename T>
__device__ __forceinline__ cx<T> acmul(cx<T> a, cx<T> b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
template <typename T>
__device__ __forceinline__ cx<T> aconj(cx<T> a) { return {a.re, -a.im}; }

// C = A B, 2x2 row-major
template <typename T>
__device__ __forceinline__ void mm2(const cx<T> *A, const cx<T> *B, cx<T> *C) {
#pragma unroll
    for (int p = 0; p < 2; p++)
#pragma unroll
        for (int q = 0; q < 2; q++) {
            cx<T> x = acmul(A[2 * p], B[q]), y = acmul(A[2 * p + 1], B[2 + q]);
            C[2 * p + q] = {x.re + y.re, x.im + y.im};
        }
}
template <typename T>
__device__ __forceinline__ void dag2(const cx<T> *A, cx<T> *B) {
    B[0] = aconj(A[0]);
    B[1] = aconj(A[2]);
    B[2] = aconj(A[1]);
    B[3] = aconj(A[3]);
}

// One thread per exact two-level molecule.  Forward: rho' = U rho U^+ with
// U = cos(W dt) - i sin(W dt)/W Z, Z = H - tr(H)/2, W^2 = z^2 + |b|^2 (the global
// phase cancels), H = H0 - Et . mu; mudot = (<mu>' - <mu>)/dt; the current scatter
// uses gamma mudot and the gather gamma sum E kappa.  Reversed here with the chain
// rule through that closed form.
template <typename T>
__global__ void adj_mol_kernel(const AdjMolArgs<T> a) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.nmol || a.kind[m] != 0) return;  // RK4 molecules: adj_rk4_kernel
    const int cmk = a.cmask[m];
    const long long o = a.off[m];
    const T gam = a.gamma[m], dt = a.dt;
    // sum of the adjoint field over the window: G_c = sum kappa U^{n+1}
    T G[3] = {T(0), T(0), T(0)};
    for (int t = a.moff[m]; t < a.moff[m + 1]; t++) {
        const T *pp = a.part + 3ll * a.mlist[t];
        G[0] += pp[0];
        G[1] += pp[1];
        G[2] += pp[2];
    }
    cx<T> mu[3][4], rho[4], R[4], H[4];
    T Et[3], md[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const bool on = (cmk >> c) & 1;
        if (!on) G[c] = T(0);
        Et[c] = a.Et_n[3 * m + c];
        md[c] = a.md_n[3 * m + c];
#pragma unroll
        for (int e = 0; e < 4; e++) mu[c][e] = on ? a.mu[c * a.pool + o + e] : cx<T>{T(0), T(0)};
    }
    // J = sum gamma mudot kappa enters E^{n+1} as -dt/eps J, so Jbar = -dt U^{n+1} and
    // mudotbar_c = gamma sum Jbar kappa = -gamma dt G_c; d/dgamma from the scatter:
    double gg = 0.0;
#pragma unroll
    for (int c = 0; c < 3; c++) gg += (double)md[c] * (double)(-dt * G[c]);
    // total adjoint of rho': incoming + gradient of mudot (grad <mu_c> = mu_c)
#pragma unroll
    for (int e = 0; e < 4; e++) {
        rho[e] = a.rho_n[o + e];
        cx<T> r = a.rhob[o + e];
        cx<T> h = a.H0[o + e];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const T f = -gam * G[c];  // mudotbar_c / dt
            r.re += f * mu[c][e].re;
            r.im += f * mu[c][e].im;
            h.re -= Et[c] * mu[c][e].re;
            h.im -= Et[c] * mu[c][e].im;
        }
        R[e] = r;
        H[e] = h;
    }
    const T z = T(0.5) * (H[0].re - H[3].re);
    const cx<T> b = H[1];
    const T W = sqrt(z * z + b.re * b.re + b.im * b.im);
    const T x = W * dt;
    const T cw = cos(x);
    const T sw = W > T(0) ? sin(x) / W : dt;
    cx<T> U[4] = {{cw, -sw * z}, {sw * b.im, -sw * b.re}, {-sw * b.im, -sw * b.re}, {cw, sw * z}};
    cx<T> Ud[4], T1[4], T2[4];
    dag2(U, Ud);
    // rhobar^n = U^+ R U - grad of <mu>(rho^n) term
    mm2(Ud, R, T1);
    mm2(T1, U, T2);
#pragma unroll
    for (int e = 0; e < 4; e++) {
        cx<T> r = T2[e];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const T f = -gam * G[c];
            r.re -= f * mu[c][e].re;
            r.im -= f * mu[c][e].im;
        }
        a.rhob[o + e] = r;
    }
    // d(sin(x)/W)/dW / W: (dt cos x - sin x / W) / W^2, series near W = 0
    const T small = sizeof(T) == 4 ? T(2e-2) : T(1e-3);
    const T fs = x < small ? dt * dt * dt * (T(-1) / T(3) + x * x / T(30)) : (dt * cw - sw) / (W * W);
    cx<T> rUd[4];
    mm2(rho, Ud, rUd);  // rho U^+
    double Etb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        Etb[c] = 0.0;
        if (!((cmk >> c) & 1)) continue;
        // dH/dEt_c = -mu_c: dz = -(mu00 - mu11)/2, db = -mu01
        const T dz = -T(0.5) * (mu[c][0].re - mu[c][3].re);
        const cx<T> dbb = {-mu[c][1].re, -mu[c][1].im};
        const T q = z * dz + b.re * dbb.re + b.im * dbb.im;  // W dW
        const T dcw = -sw * dt * q;
        const T dsw = fs * q;
        // dU = dcw - i (dsw Z + sw dZ), Z = [[z, b], [conj b, -z]]
        const cx<T> Z[4] = {{z, T(0)}, b, aconj(b), {-z, T(0)}};
        const cx<T> dZ[4] = {{dz, T(0)}, dbb, aconj(dbb), {-dz, T(0)}};
        cx<T> dU[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const T mr = dsw * Z[e].re + sw * dZ[e].re, mi = dsw * Z[e].im + sw * dZ[e].im;
            dU[e] = {mi, -mr};  // -i (mr + i mi)
            if (e == 0 || e == 3) dU[e].re += dcw;
        }
        // P = dU rho U^+ + U rho dU^+ = X + X^+ with X = dU rho U^+
        cx<T> X[4];
        mm2(dU, rUd, X);
        double s = 0.0;
#pragma unroll
        for (int p = 0; p < 2; p++)
#pragma unroll
            for (int qq = 0; qq < 2; qq++) {
                const cx<T> xv = X[2 * p + qq], xt = aconj(X[2 * qq + p]);
                const cx<T> r = R[2 * p + qq];
                s += (double)r.re * ((double)xv.re + (double)xt.re) + (double)r.im * ((double)xv.im + (double)xt.im);
            }
        Etb[c] = s;
    }
    // Et = gamma sum E^n kappa: d/dgamma = Etbar . Et / gamma; scatter amplitude
#pragma unroll
    for (int c = 0; c < 3; c++) {
        gg += Etb[c] * (double)Et[c] / (double)gam;
        a.cadj[3 * m + c] = (T)(-(double)gam * Etb[c] / (double)dt);
    }
    a.ggam[m] += gg;
}

// ------------------------------------------------------------------ RK4 GKSL molecules
// Reverse of one molecule step of nsub classic RK4 substeps of the GKSL equation under
// the held H = H0 - Et . mu (one warp per molecule; lane owns elements lane and lane +
// 32 of the row-major n x n matrices, which live in shared memory).  With Y the adjoint
// of a substep's result and rho_s its start, the stages S2 = rho_s + h/2 k1, S3 =
// rho_s + h/2 k2, S4 = rho_s + h k3 (k = L(S)) are recomputed, then walked back:
//   kb4 = h/6 Y, kb3 = h/3 Y, kb2 = h/3 Y, kb1 = h/6 Y, rhob = Y,
//   Sb = L^+(kb4): rhob += Sb, kb3 += h Sb;   Sb = L^+(kb3): rhob += Sb, kb2 += h/2 Sb;
//   Sb = L^+(kb2): rhob += Sb, kb1 += h/2 Sb; rhob += L^+(kb1),
// and Etb_c += Re<kb, dL/dEt_c (S)> at each stage, dL/dEt_c (S) = i [mu_c, S].  Under the
// inner product Re Tr(X^+ Y), L^+(X) = i [H, X] + D^+(X): the ladder decay moves
// population down in D and up in D^+ (element (j, j) gains decay X_{j-1,j-1}); the
// dephasing part is self-adjoint.  rho_s is rebuilt from rho^n by s forward substeps.
constexpr int ADJ_RK4_WARPS = 4;

template <typename T>
struct AdjRk4Shared {
    cx<T> H[ADJ_RK4_WARPS][64];
    cx<T> Mu[ADJ_RK4_WARPS][3][64];
    cx<T> S[ADJ_RK4_WARPS][4][64];  // rho_s, S2, S3, S4
    cx<T> K[ADJ_RK4_WARPS][64];     // argument of the next L or L^+
};

template <typename T>
__device__ __forceinline__ T warp_sum_adj(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// L(S)_jl (the forward GKSL right-hand side of the molecule kernel)
template <typename T>
__device__ __forceinline__ cx<T> gksl(int n, int j, int l, const cx<T> *S, const cx<T> *H, T decay, T deph) {
    cx<T> acc = {T(0), T(0)};
    for (int p = 0; p < n; p++) {
        const cx<T> x = acmul(H[j * n + p], S[p * n + l]), y = acmul(S[j * n + p], H[p * n + l]);
        acc.re += x.re - y.re;
        acc.im += x.im - y.im;
    }
    cx<T> out = {acc.im, -acc.re};  // -i acc
    const cx<T> r = S[j * n + l];
    const T f = T(0.5) * decay * (T(j >= 1) + T(l >= 1));
    out.re -= f * r.re;
    out.im -= f * r.im;
    if (j == l && j + 1 < n) out.re += decay * S[(j + 1) * n + (j + 1)].re;
    if (j != l) {
        out.re -= deph * r.re;
        out.im -= deph * r.im;
    }
    return out;
}

// L^+(X)_jl
template <typename T>
__device__ __forceinline__ cx<T> gksl_adj(int n, int j, int l, const cx<T> *X, const cx<T> *H, T decay, T deph) {
    cx<T> acc = {T(0), T(0)};
    for (int p = 0; p < n; p++) {
        const cx<T> x = acmul(H[j * n + p], X[p * n + l]), y = acmul(X[j * n + p], H[p * n + l]);
        acc.re += x.re - y.re;
        acc.im += x.im - y.im;
    }
    cx<T> out = {-acc.im, acc.re};  // +i acc
    const cx<T> r = X[j * n + l];
    const T f = T(0.5) * decay * (T(j >= 1) + T(l >= 1));
    out.re -= f * r.re;
    out.im -= f * r.im;
    if (j == l && j >= 1) out.re += decay * X[(j - 1) * n + (j - 1)].re;
    if (j != l) {
        out.re -= deph * r.re;
        out.im -= deph * r.im;
    }
    return out;
}

// Re( conj(Y_jl) (i [mu, S])_jl )
template <typename T>
__device__ __forceinline__ T dl_dot(int n, int j, int l, cx<T> y, const cx<T> *Mu, const cx<T> *S) {
    cx<T> acc = {T(0), T(0)};
    for (int p = 0; p < n; p++) {
        const cx<T> x = acmul(Mu[j * n + p], S[p * n + l]), z = acmul(S[j * n + p], Mu[p * n + l]);
        acc.re += x.re - z.re;
        acc.im += x.im - z.im;
    }
    const cx<T> d = {-acc.im, acc.re};  // i acc
    return y.re * d.re + y.im * d.im;
}

template <typename T>
__global__ void __launch_bounds__(ADJ_RK4_WARPS * 32) adj_rk4_kernel(const AdjMolArgs<T> a) {
    __shared__ AdjRk4Shared<T> sh;
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int m = blockIdx.x * ADJ_RK4_WARPS + wl;
    if (m >= a.nmol || a.kind[m] == 0) return;  // whole warp
    const int n = a.nlev[m], nn = n * n, ns = a.nsub[m];
    const int cmk = a.cmask[m];
    const long long o = a.off[m];
    const T gam = a.gamma[m], dt = a.dt, h = dt / T(ns), decay = a.decay[m], deph = a.dephase[m];
    cx<T> *H = sh.H[wl], *K = sh.K[wl];
    cx<T> *Rs = sh.S[wl][0], *S2 = sh.S[wl][1], *S3 = sh.S[wl][2], *S4 = sh.S[wl][3];
    // G_c = sum kappa U^{n+1} (the molecule's gather partials, lane-strided, fixed tree)
    T G[3] = {T(0), T(0), T(0)};
    for (int t = a.moff[m] + lane; t < a.moff[m + 1]; t += 32) {
        const T *pp = a.part + 3ll * a.mlist[t];
        G[0] += pp[0];
        G[1] += pp[1];
        G[2] += pp[2];
    }
    T Et[3], md[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        G[c] = ((cmk >> c) & 1) ? warp_sum_adj(G[c]) : T(0);
        Et[c] = a.Et_n[3 * m + c];
        md[c] = a.md_n[3 * m + c];
    }
    int jj[2], ll[2];
    bool own[2];
    cx<T> Y[2], r0[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const int e = lane + 32 * q;
        own[q] = e < nn;
        jj[q] = own[q] ? e / n : 0;
        ll[q] = own[q] ? e - jj[q] * n : 0;
        if (own[q]) {
            cx<T> hv = a.H0[o + e];
            cx<T> y = a.rhob[o + e];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const cx<T> mv = ((cmk >> c) & 1) ? a.mu[c * a.pool + o + e] : cx<T>{T(0), T(0)};
                sh.Mu[wl][c][e] = mv;
                hv.re -= Et[c] * mv.re;
                hv.im -= Et[c] * mv.im;
                // adjoint of rho' gains the gradient of mudot: (-gamma G_c) mu_c
                y.re += -gam * G[c] * mv.re;
                y.im += -gam * G[c] * mv.im;
            }
            H[e] = hv;
            Y[q] = y;
            r0[q] = a.rho_n[o + e];
        }
    }
    __syncwarp();
    double Etb[3] = {0.0, 0.0, 0.0};
    T eb[3] = {T(0), T(0), T(0)};
    for (int sidx = ns - 1; sidx >= 0; sidx--) {
        // rho_s: sidx forward substeps from rho^n
#pragma unroll
        for (int q = 0; q < 2; q++)
            if (own[q]) Rs[lane + 32 * q] = r0[q];
        __syncwarp();
        for (int f = 0; f <= sidx; f++) {
            // stages of substep f from Rs (kept in S2, S3, S4); for f < sidx also its result
            cx<T> base[2], acc[2] = {{T(0), T(0)}, {T(0), T(0)}}, kk[2];
#pragma unroll
            for (int q = 0; q < 2; q++) base[q] = own[q] ? Rs[lane + 32 * q] : cx<T>{T(0), T(0)};
            const cx<T> *src = Rs;
            cx<T> *dsts[3] = {S2, S3, S4};
#pragma unroll
            for (int st = 0; st < 4; st++) {
                const T wgt = (st == 0 || st == 3) ? T(1) : T(2);
#pragma unroll
                for (int q = 0; q < 2; q++)
                    if (own[q]) {
                        kk[q] = gksl(n, jj[q], ll[q], src, H, decay, deph);
                        acc[q].re += wgt * kk[q].re;
                        acc[q].im += wgt * kk[q].im;
                    }
                if (st < 3) {
                    const T cn = st < 2 ? T(0.5) : T(1);
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        if (own[q]) dsts[st][lane + 32 * q] = {base[q].re + cn * h * kk[q].re, base[q].im + cn * h * kk[q].im};
                    __syncwarp();
                    src = dsts[st];
                }
            }
            if (f < sidx) {
                __syncwarp();
#pragma unroll
                for (int q = 0; q < 2; q++)
                    if (own[q]) Rs[lane + 32 * q] = {base[q].re + h / T(6) * acc[q].re, base[q].im + h / T(6) * acc[q].im};
                __syncwarp();
            }
        }
        // walk the stages of substep sidx back
        cx<T> rb[2], kb[2];
        auto put_k = [&](const cx<T> (&v)[2]) {
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 2; q++)
                if (own[q]) K[lane + 32 * q] = v[q];
            __syncwarp();
        };
        auto dots = [&](const cx<T> (&v)[2], const cx<T> *Sst) {
#pragma unroll
            for (int c = 0; c < 3; c++)
                if ((cmk >> c) & 1)
#pragma unroll
                    for (int q = 0; q < 2; q++)
                        if (own[q]) eb[c] += dl_dot(n, jj[q], ll[q], v[q], sh.Mu[wl][c], Sst);
        };
        cx<T> k3b[2], k2b[2], k1b[2], sb[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            rb[q] = Y[q];
            kb[q] = {h / T(6) * Y[q].re, h / T(6) * Y[q].im};  // kb4
            k3b[q] = {h / T(3) * Y[q].re, h / T(3) * Y[q].im};
            k2b[q] = k3b[q];
            k1b[q] = kb[q];
        }
        // k4 = L(S4), S4 = rho_s + h k3
        put_k(kb);
        dots(kb, S4);
#pragma unroll
        for (int q = 0; q < 2; q++)
            if (own[q]) {
                sb[q] = gksl_adj(n, jj[q], ll[q], K, H, decay, deph);
                rb[q].re += sb[q].re; rb[q].im += sb[q].im;
                k3b[q].re += h * sb[q].re; k3b[q].im += h * sb[q].im;
            }
        // k3 = L(S3), S3 = rho_s + h/2 k2
        put_k(k3b);
        dots(k3b, S3);
#pragma unroll
        for (int q = 0; q < 2; q++)
            if (own[q]) {
                sb[q] = gksl_adj(n, jj[q], ll[q], K, H, decay, deph);
                rb[q].re += sb[q].re; rb[q].im += sb[q].im;
                k2b[q].re += T(0.5) * h * sb[q].re; k2b[q].im += T(0.5) * h * sb[q].im;
            }
        // k2 = L(S2), S2 = rho_s + h/2 k1
        put_k(k2b);
        dots(k2b, S2);
#pragma unroll
        for (int q = 0; q < 2; q++)
            if (own[q]) {
                sb[q] = gksl_adj(n, jj[q], ll[q], K, H, decay, deph);
                rb[q].re += sb[q].re; rb[q].im += sb[q].im;
                k1b[q].re += T(0.5) * h * sb[q].re; k1b[q].im += T(0.5) * h * sb[q].im;
            }
        // k1 = L(rho_s)
        put_k(k1b);
        dots(k1b, Rs);
#pragma unroll
        for (int q = 0; q < 2; q++)
            if (own[q]) {
                sb[q] = gksl_adj(n, jj[q], ll[q], K, H, decay, deph);
                Y[q] = {rb[q].re + sb[q].re, rb[q].im + sb[q].im};
            }
        __syncwarp();
    }
    // adjoint of rho^n: the reversed steps, minus the gradient of <mu>(rho^n) in mudot
#pragma unroll
    for (int q = 0; q < 2; q++)
        if (own[q]) {
            const int e = lane + 32 * q;
            cx<T> r = Y[q];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const cx<T> mv = sh.Mu[wl][c][e];
                r.re -= -gam * G[c] * mv.re;
                r.im -= -gam * G[c] * mv.im;
            }
            a.rhob[o + e] = r;
        }
#pragma unroll
    for (int c = 0; c < 3; c++) Etb[c] = (double)warp_sum_adj(eb[c]);
    if (lane == 0) {
        double gg = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            gg += (double)md[c] * (double)(-dt * G[c]);
            gg += Etb[c] * (double)Et[c] / (double)gam;
            a.cadj[3 * m + c] = (T)(-(double)gam * Etb[c] / (double)dt);
        }
        a.ggam[m] += gg;
    }
}

// Copy what the reverse sweep needs from one forward step: the design-box E (3 x
// nbox), rho (pool) and, if rec_mol, the step's field and mudot (3 per molecule).
template <typename T>
__global__ void adj_record_kernel(const T *E0, const T *E1, const T *E2, int px, long long plane, int bx0, int by0,
                                  int bz0, int bsx, int bsy, long long nbox, T *recE, const cx<T> *rho, long long pool,
                                  cx<T> *recRho, const T *Et, const T *md, int nmol3, T *recEt, T *recMd) {
    const long long total = 3 * nbox + pool + nmol3;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < 3 * nbox) {
            const int c = (int)(t / nbox);
            const long long q = t % nbox;
            const int i = (int)(q % bsx), j = (int)((q / bsx) % bsy), k = (int)(q / ((long long)bsx * bsy));
            const T *E = c == 0 ? E0 : (c == 1 ? E1 : E2);
            recE[t] = E[(long long)(bz0 + k + 1) * plane + (long long)(by0 + j + 1) * px + (bx0 + i + XO)];
        } else if (t < 3 * nbox + pool) {
            recRho[t - 3 * nbox] = rho[t - 3 * nbox];
        } else if (recEt) {
            const long long q = t - 3 * nbox - pool;
            recEt[q] = Et[q];
            recMd[q] = md[q];
        }
    }
}

// ------------------------------------------------------------------ host driver

namespace {

// work memory of one call, from the process allocator, returned when the call ends
ml_status adj_alloc(DevList &L, void **out, size_t bytes) { return dev_alloc(L.v, out, bytes); }

#define AA(ptr, bytes)                                             \
    do {                                                           \
        ml_status s_ = adj_alloc(L, (void **)&(ptr), (bytes));     \
        if (s_ != ML_OK) return s_;                                \
    } while (0)

struct Snap {
    long long step;
    int nsamp;
    long long samp_step0;
};

ml_status snapshot(ml_grid *g, char *dst, Snap &sn, cudaStream_t s) {
    for (auto &b : state_blobs(g)) {
        CK(cudaMemcpyAsync(dst, b.p, b.bytes, cudaMemcpyDeviceToDevice, s));
        dst += b.bytes;
    }
    sn = {g->step, g->nsamp, g->samp_step0};
    return ML_OK;
}

ml_status restore(ml_grid *g, const char *src, const Snap &sn, cudaStream_t s) {
    for (auto &b : state_blobs(g)) {
        CK(cudaMemcpyAsync(b.p, src, b.bytes, cudaMemcpyDeviceToDevice, s));
        src += b.bytes;
    }
    g->step = sn.step;
    g->nsamp = sn.nsamp;
    g->samp_step0 = sn.samp_step0;
    return ML_OK;
}

template <typename T>
ml_status adjoint_impl(ml_grid *g, long long N, int K, int pid, int f, double *obj, double *grad_eps,
                       double *grad_gamma, int on_device, cudaStream_t s) {
    DevList L;
    const Plane &pl = g->planes[pid];
    const long long ncell = (long long)pl.nb * pl.nc;
    const int M = g->nmol;
    bool any_rk4 = false;  // RK4 GKSL molecules take their own reverse kernel
    for (int m = 0; m < M; m++) any_rk4 = any_rk4 || g->kind[m] != 0;
    const long long nbox = g->dcb ? (long long)g->dbox[3] * g->dbox[4] * g->dbox[5] : 0;
    // the objective counts the steps of this run only
    CK(cudaGetLastError());
    {
        ml_status st = fold_planes<T>(g, s);
        if (st != ML_OK) return st;
    }
    CK(cudaMemsetAsync(pl.d_acc, 0, 4 * (size_t)pl.nfreq * ncell * sizeof(double2), s));
    if (!grad_eps && !grad_gamma) {
        // no gradient wanted: the forward steps and the objective only
        ml_status st = step_impl<T>(g, N, s);
        if (st == ML_OK) st = fold_planes<T>(g, s);
        if (st != ML_OK) return st;
        CK(launch_flux_reduce(pl.d_acc, (int)ncell, pl.nfreq, g->d_fpart, g->d_scalar, s));
        double objv = 0.0;
        CK(cudaMemcpyAsync(&objv, g->d_scalar + f, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (obj) *obj = objv;
        return ML_OK;
    }
    const long long n0 = g->step;
    // ---- forward sweep with a full-state checkpoint at the start of every segment
    size_t sbytes = 0;
    for (auto &b : state_blobs(g)) sbytes += b.bytes;
    const long long nseg = (N + K - 1) / K;
    char *ck = nullptr;
    AA(ck, sbytes * (size_t)(nseg + 1));
    std::vector<Snap> snaps(nseg + 1);
    for (long long sg = 0; sg < nseg; sg++) {
        ml_status st = snapshot(g, ck + sbytes * sg, snaps[sg], s);
        if (st != ML_OK) return st;
        st = step_impl<T>(g, std::min<long long>(K, N - sg * K), s);
        if (st != ML_OK) return st;
    }
    {
        ml_status st = fold_planes<T>(g, s);
        if (st != ML_OK) return st;
        st = snapshot(g, ck + sbytes * nseg, snaps[nseg], s);
        if (st != ML_OK) return st;
    }
    CK(launch_flux_reduce(pl.d_acc, (int)ncell, pl.nfreq, g->d_fpart, g->d_scalar, s));
    // the chosen frequency's sums, kept aside: the recompute below refills the plane
    double2 *objacc = nullptr;
    AA(objacc, 4 * (size_t)ncell * sizeof(double2));
    for (int q = 0; q < 4; q++)
        CK(cudaMemcpyAsync(objacc + q * ncell, pl.d_acc + ((long long)q * pl.nfreq + f) * ncell,
                           ncell * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    double objv = 0.0;
    CK(cudaMemcpyAsync(&objv, g->d_scalar + f, sizeof(double), cudaMemcpyDeviceToHost, s));
    // ---- adjoint state
    const size_t esz = sizeof(T);
    T *U[3], *Hb[3];
    for (int c = 0; c < 3; c++) {
        AA(U[c], g->vol * esz);
        AA(Hb[c], g->vol * esz);
        CK(cudaMemsetAsync(U[c], 0, g->vol * esz, s));
        CK(cudaMemsetAsync(Hb[c], 0, g->vol * esz, s));
    }
    T *phi[2][3][2] = {}, *chi[2][3][2] = {};
    for (int a = 0; a < 3; a++)
        if (g->psi_n[a])
            for (int q = 0; q < 2; q++)
                for (int l = 0; l < 2; l++) {
                    AA(phi[l][a][q], g->psi_n[a] * esz);
                    AA(chi[l][a][q], g->psi_n[a] * esz);
                    CK(cudaMemsetAsync(phi[l][a][q], 0, g->psi_n[a] * esz, s));
                    CK(cudaMemsetAsync(chi[l][a][q], 0, g->psi_n[a] * esz, s));
                }
    T *JDb = nullptr, *PDb = nullptr;  // adjoints of the pole currents and polarisations
    if (g->JD) {
        const size_t cnt = 3 * (size_t)g->npole * g->jcnt;
        AA(JDb, cnt * esz);
        CK(cudaMemsetAsync(JDb, 0, cnt * esz, s));
        if (g->PD) {
            AA(PDb, cnt * esz);
            CK(cudaMemsetAsync(PDb, 0, cnt * esz, s));
        }
    }
    double *geps = nullptr, *ggam = nullptr;
    T *gseg = nullptr;
    if (nbox) {
        AA(geps, nbox * sizeof(double));
        CK(cudaMemsetAsync(geps, 0, nbox * sizeof(double), s));
        AA(gseg, nbox * esz);
        CK(cudaMemsetAsync(gseg, 0, nbox * esz, s));
    }
    cx<T> *rhob = nullptr;
    T *cadj = nullptr;
    if (M) {
        AA(ggam, M * sizeof(double));
        CK(cudaMemsetAsync(ggam, 0, M * sizeof(double), s));
        AA(rhob, (size_t)g->pool * sizeof(cx<T>));
        CK(cudaMemsetAsync(rhob, 0, (size_t)g->pool * sizeof(cx<T>), s));
        AA(cadj, 3 * (size_t)M * esz);
    }
    // per-segment records: slot t holds E^n (design box) and rho^n of step n = seg0 + t,
    // and (t >= 1) the field and mudot of step n - 1
    const size_t slotE = 3 * (size_t)nbox, slotR = (size_t)g->pool, slotM = 3 * (size_t)M;
    T *recE = nullptr, *recEt = nullptr, *recMd = nullptr;
    cx<T> *recR = nullptr;
    AA(recE, (size_t)(K + 1) * slotE * esz);
    if (M) {
        AA(recR, (size_t)(K + 1) * slotR * sizeof(cx<T>));
        AA(recEt, (size_t)(K + 1) * slotM * esz);
        AA(recMd, (size_t)(K + 1) * slotM * esz);
    }
    // ---- field-pass arguments shared by every reversed step
    AdjFieldArgs<T> fa{};
    fa.nx = g->nx; fa.ny = g->ny; fa.nz = g->nz; fa.px = g->px; fa.plane = g->plane;
    for (int a = 0; a < 3; a++) fa.per[a] = g->per[a];
    for (int q = 0; q < 6; q++) fa.pml[q] = g->pml[q];
    fa.dt = (T)g->dt;
    for (int c = 0; c < 3; c++) { fa.U[c] = U[c]; fa.Hb[c] = Hb[c]; fa.cpml[c] = (const T *)g->cpml[c]; }
    fa.JDb = JDb;
    fa.PDb = PDb;
    fa.npole = g->npole;
    fa.jcnt = (long long)g->jcnt;
    fa.mat = g->mat;
    fa.mat_cb = (const T *)g->mat_cb; fa.mat_dk = (const T *)g->mat_dk; fa.mat_db = (const T *)g->mat_db;
    fa.mat_dp = (const T *)g->mat_dp;
    for (int q = 0; q < 6; q++) { fa.dbox[q] = g->dbox[q]; fa.jbox[q] = g->jbox[q]; }
    fa.dcb = (const T *)g->dcb;
    if (M)
        for (int a = 0; a < 3; a++) {
            fa.jb0[a] = g->jb0[a];
            fa.jbn[a] = g->jbn[a];
            fa.Jb[a] = (const T *)g->d_J[a];
        }
    fa.gseg = gseg;
    fa.nbox = nbox;
    fa.pax = pl.axis; fa.pidx = pl.index; fa.pnb = pl.nb;
    {
        const int nax = pl.axis == 0 ? g->nx : (pl.axis == 1 ? g->ny : g->nz);
        fa.pim = pl.index - 1;
        fa.hasm = 1;
        if (fa.pim < 0) {
            if (g->per[pl.axis]) fa.pim += nax;
            else fa.hasm = 0;
        }
    }
    cx<T> *tab = nullptr;
    AA(tab, 4 * (size_t)ncell * sizeof(cx<T>));
    adj_table_kernel<T><<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(objacc, ncell, g->dt, tab);
    CK(cudaGetLastError());
    g->launches++;
    fa.tab = tab;
    const double omega = pl.omega[f];
    auto phase = [&](double t, T &cs, T &sn) {
        cs = (T)std::cos(omega * t);
        sn = (T)std::sin(omega * t);
    };
    const dim3 fgrid((g->nx + 31) / 32, (g->ny + 7) / 8, (g->nz + AZC - 1) / AZC), fblock(32, 8);
    // d objective / d E^N
    phase((double)(n0 + N) * g->dt, fa.csE, fa.snE);
    adj_inject_kernel<T><<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(fa, pl.nc);
    CK(cudaGetLastError());
    g->launches++;
    int ping = 0;
    struct Ev {
        cudaEvent_t e = nullptr;
        ~Ev() {
            if (e) cudaEventDestroy(e);
        }
    } ev_fork, ev_join;
    const cudaStream_t cs = (M && g->side) ? g->side : s;
    if (M) {
        CK(cudaEventCreateWithFlags(&ev_fork.e, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ev_join.e, cudaEventDisableTiming));
    }
    for (long long sg = nseg - 1; sg >= 0; sg--) {
        const long long seg0 = sg * K, len = std::min<long long>(K, N - seg0);
        ml_status st = restore(g, ck + sbytes * sg, snaps[sg], s);
        if (st != ML_OK) return st;
        auto record = [&](long long slot, bool mol) -> ml_status {
            const int cur = g->cur;
            const long long total = 3 * nbox + (M ? g->pool : 0) + (mol && M ? 3 * M : 0);
            if (total == 0) return ML_OK;
            const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 4096);
            adj_record_kernel<T><<<blocks, 256, 0, s>>>(
                (const T *)g->F[cur][0], (const T *)g->F[cur][1], (const T *)g->F[cur][2], g->px, g->plane, g->dbox[0],
                g->dbox[1], g->dbox[2], g->dbox[3] ? g->dbox[3] : 1, g->dbox[4] ? g->dbox[4] : 1, nbox,
                recE + slot * slotE, M ? (const cx<T> *)g->d_rho : nullptr, M ? g->pool : 0,
                recR ? recR + slot * slotR : nullptr, (const T *)g->d_Et, (const T *)g->d_mudot,
                (mol && M) ? 3 * M : 0, (mol && M) ? recEt + slot * slotM : nullptr,
                (mol && M) ? recMd + slot * slotM : nullptr);
            CK(cudaGetLastError());
            g->launches++;
            return ML_OK;
        };
        st = record(0, false);
        if (st != ML_OK) return st;
        for (long long t = 0; t < len; t++) {
            st = step_impl<T>(g, 1, s);
            if (st != ML_OK) return st;
            st = record(t + 1, true);
            if (st != ML_OK) return st;
        }
        for (long long t = len - 1; t >= 0; t--) {
            const long long n = seg0 + t;
            if (M) {
                // the molecule chain of this step runs on the side stream beside pass A
                // (pass A reads only U, Hbar and phi); pass B waits for its current
                CK(cudaEventRecord(ev_fork.e, s));
                CK(cudaStreamWaitEvent(cs, ev_fork.e, 0));
                GathArgs<T> ga{};
                ga.nblocks = g->jnb; ga.nbx = g->jnbx; ga.nby = g->jnby;
                for (int q = 0; q < 3; q++) { ga.bn[q] = g->jbn[q]; ga.b0[q] = g->jb0[q]; ga.E[q] = U[q]; }
                ga.px = g->px; ga.plane = g->plane;
                ga.off = g->d_joff; ga.ent = g->d_jent; ga.wf = g->d_wf; ga.w = (const T *)g->d_w; ga.cmask = g->d_cmask;
                ga.gcmask = g->gcmask; ga.part = (T *)g->d_part;
                CK(launch_gather<T>(ga, cs));
                g->launches++;
                AdjMolArgs<T> ma{};
                ma.nmol = M; ma.dt = (T)g->dt; ma.cmask = g->d_cmask; ma.off = g->d_off;
                ma.gamma = (const T *)g->d_gamma; ma.H0 = (const cx<T> *)g->d_H0; ma.mu = (const cx<T> *)g->d_mu;
                ma.pool = g->pool; ma.moff = g->d_moff; ma.mlist = g->d_mlist; ma.part = (const T *)g->d_part;
                ma.rho_n = recR + t * slotR; ma.Et_n = recEt + (t + 1) * slotM; ma.md_n = recMd + (t + 1) * slotM;
                ma.rhob = rhob; ma.cadj = cadj; ma.ggam = ggam;
                ma.kind = g->d_kind; ma.nlev = g->d_nlev; ma.nsub = g->d_nsub;
                ma.decay = (const T *)g->d_decay; ma.dephase = (const T *)g->d_deph;
                adj_mol_kernel<T><<<(M + 127) / 128, 128, 0, cs>>>(ma);
                if (any_rk4) {
                    adj_rk4_kernel<T><<<(M + ADJ_RK4_WARPS - 1) / ADJ_RK4_WARPS, ADJ_RK4_WARPS * 32, 0, cs>>>(ma);
                    g->launches++;
                }
                CK(cudaGetLastError());
                g->launches++;
                CurArgs<T> ca;
                fill_cur_args<T>(g, ca);
                ca.c = cadj;
                CK(launch_current<T>(ca, cs));
                g->launches++;
                CK(cudaEventRecord(ev_join.e, cs));
            }
            for (int a = 0; a < 3; a++)
                for (int q = 0; q < 2; q++) {
                    fa.phi_in[a][q] = phi[ping][a][q];
                    fa.phi_out[a][q] = phi[ping ^ 1][a][q];
                    fa.chi_in[a][q] = chi[ping][a][q];
                    fa.chi_out[a][q] = chi[ping ^ 1][a][q];
                }
            fa.Eprev = recE + t * slotE;
            fa.Enext = recE + (t + 1) * slotE;
            phase(((double)(n0 + n) + 0.5) * g->dt, fa.csH, fa.snH);
            phase((double)(n0 + n) * g->dt, fa.csE, fa.snE);
            fa.injectE = n >= 1;
            adj_passA_kernel<T><<<fgrid, fblock, 0, s>>>(fa);
            CK(cudaGetLastError());
            if (M) CK(cudaStreamWaitEvent(s, ev_join.e, 0));
            adj_passB_kernel<T><<<fgrid, fblock, 0, s>>>(fa);
            CK(cudaGetLastError());
            g->launches += 2;
            ping ^= 1;
        }
        if (nbox) {
            adj_fold_kernel<T><<<(unsigned)((nbox + 255) / 256), 256, 0, s>>>(gseg, geps, nbox);
            CK(cudaGetLastError());
            g->launches++;
        }
    }
    // ---- results, and the forward end state back in place
    if (grad_eps && nbox)
        CK(cudaMemcpyAsync(grad_eps, geps, nbox * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (grad_gamma && M)
        CK(cudaMemcpyAsync(grad_gamma, ggam, M * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    {
        ml_status st = restore(g, ck + sbytes * nseg, snaps[nseg], s);
        if (st != ML_OK) return st;
    }
    CK(cudaStreamSynchronize(s));
    if (obj) *obj = objv;
    return ML_OK;
}

}  // namespace
}  // namespace ml

using namespace ml;

ml_status ml_adjoint_run(ml_grid *g, int64_t nsteps, int ckpt_every, int plane_id, int freq, double *objective,
                         double *grad_eps, double *grad_gamma, int on_device, void *stream) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    if (nsteps < 1 || ckpt_every < 1) return fail(ML_ERR_INVALID_ARG, "nsteps and ckpt_every must be >= 1");
    if (plane_id < 0 || plane_id >= (int)g->planes.size()) return fail(ML_ERR_INVALID_ARG, "no such plane");
    if (freq < 0 || freq >= g->planes[plane_id].nfreq) return fail(ML_ERR_INVALID_ARG, "no such frequency");
    if (grad_eps && !g->dcb) return fail(ML_ERR_INVALID_ARG, "grad_eps needs a design box");
    for (int m = 0; m < g->nmol; m++)
        if (g->gamma[m] == 0.0) return fail(ML_ERR_INVALID_ARG, "the adjoint needs gamma != 0 for every molecule");
    const int K = (int)std::min<int64_t>(ckpt_every, nsteps);
    cudaStream_t s = (cudaStream_t)stream;
    g->pop_off = true;  // the sweeps write no population sink
    const ml_status st =
        g->prec ? adjoint_impl<double>(g, nsteps, K, plane_id, freq, objective, grad_eps, grad_gamma, on_device, s)
                : adjoint_impl<float>(g, nsteps, K, plane_id, freq, objective, grad_eps, grad_gamma, on_device, s);
    g->pop_off = false;
    return st;
}

// Parameters of the objective: the design-box permittivity and the couplings.
ml_status ml_set_design_eps(ml_grid *g, const double *eps, int on_device, void *stream) {
    if (!g || !eps) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (!g->dcb) return fail(ML_ERR_INVALID_ARG, "the grid has no design box");
    const size_t n = (size_t)g->dbox[3] * g->dbox[4] * g->dbox[5];
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> v(n);
    if (on_device) {
        CK(cudaMemcpyAsync(v.data(), eps, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        std::copy(eps, eps + n, v.begin());
    }
    for (size_t q = 0; q < n; q++) {
        if (!(v[q] > 0.0)) return fail(ML_ERR_INVALID_ARG, "design eps must be > 0");
        v[q] = g->dt / v[q];
    }
    CK(cudaStreamSynchronize(s));
    if (g->prec) {
        CK(cudaMemcpy(g->dcb, v.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        CK(cudaMemcpy(g->dcb, f.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    return ML_OK;
}

ml_status ml_set_couplings(ml_grid *g, const double *gamma, int on_device, void *stream) {
    if (!g || !gamma) return fail(ML_ERR_INVALID_ARG, "null argument");
    const size_t n = (size_t)g->nmol;
    if (n == 0) return ML_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> v(n);
    if (on_device) {
        CK(cudaMemcpyAsync(v.data(), gamma, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        std::copy(gamma, gamma + n, v.begin());
    }
    for (size_t q = 0; q < n; q++)
        if (!std::isfinite(v[q])) return fail(ML_ERR_INVALID_ARG, "non-finite coupling");
    CK(cudaStreamSynchronize(s));
    if (g->prec) {
        CK(cudaMemcpy(g->d_gamma, v.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        std::vector<float> f(v.begin(), v.end());
        CK(cudaMemcpy(g->d_gamma, f.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    }
    g->gamma = v;
    return ML_OK;
}
