// K1: one fused pass per time step over the Yee grid.
//
// For a tile of TX x TY columns and a chunk of z planes, the block marches up in
// z.  At plane k it computes H^{n+1/2}(k) on the tile plus a one-cell halo on the
// low x and y sides (recomputed from E^n and H^{n-1/2}, so no other block's
// output is needed), then E^{n+1}(k) from H^{n+1/2} at k and k-1 (Eq. Maxwell,
// Yee staggering), with
//   * CPML (Roden-Gedney recursive convolution, Taflove & Hagness Ch. 7) on the
//     curl terms whose derivative runs across a layer,
//   * the per-cell coefficient dt/eps (Eq. Dromega; material table or design box),
//   * the Drude auxiliary current in Drude cells,
//   * soft current-sheet sources,
//   * the molecular current J = sum_m gamma_m mudot_m kappa_m (Eq. J_mol with
//     Eq. Polarization_mol), summed per cell in the fixed order of the tile's
//     binned molecule list (deterministic, no atomics).
// E and H are read from one time level and written to the other, so tiles never
// race.  E^n planes are staged in shared memory (k and k+1 with halo); H^{n+1/2}
// of plane k with its low halo lives in shared memory for the E update, the own
// column's H^{n+1/2}(k-1) in registers.
#include "ml_internal.cuh"

namespace ml {

template <typename T>
__device__ __forceinline__ long long gi(const YeeArgs<T> &a, int i, int j, int k) {
    return (long long)(k + 1) * a.plane + (long long)(j + 1) * a.px + (i + XO);
}

__device__ __forceinline__ int canon(int p, int n, int per) {
    if (p < 0) return per ? p + n : 0;
    if (p >= n) return per ? p - n : n - 1;
    return p;
}

// slab coordinate of canonical position p along an axis with layers lo/hi, or -1
__device__ __forceinline__ int slab(int p, int n, int lo, int hi) {
    if (p < lo) return p;
    if (p >= n - hi) return p - (n - hi) + lo;
    return -1;
}

// Write v at (i,j,k) and at every periodic ghost image of that cell.
template <typename T>
__device__ __forceinline__ void store_img(const YeeArgs<T> &a, T *f, int i, int j, int k, T v) {
    f[gi(a, i, j, k)] = v;
    bool bx = a.per[0] && (i == 0 || i == a.nx - 1);
    bool by = a.per[1] && (j == 0 || j == a.ny - 1);
    bool bz = a.per[2] && (k == 0 || k == a.nz - 1);
    if (!(bx | by | bz)) return;
    int xs[3], ys[3], zs[3];
    int nxs = 1, nys = 1, nzs = 1;
    xs[0] = i; ys[0] = j; zs[0] = k;
    if (bx) { if (i == 0) xs[nxs++] = a.nx; if (i == a.nx - 1) xs[nxs++] = -1; }
    if (by) { if (j == 0) ys[nys++] = a.ny; if (j == a.ny - 1) ys[nys++] = -1; }
    if (bz) { if (k == 0) zs[nzs++] = a.nz; if (k == a.nz - 1) zs[nzs++] = -1; }
    for (int c = 0; c < nzs; c++)
        for (int b = 0; b < nys; b++)
            for (int q = 0; q < nxs; q++)
                if (q | b | c) f[gi(a, xs[q], ys[b], zs[c])] = v;
}

// H^{n+1/2} at (i,j,k) from E^n values around it (Eq. Maxwell b) with CPML.
// hx,hy,hz: in = H^{n-1/2}, out = H^{n+1/2}.  `own`: write CPML memory.
template <typename T>
__device__ __forceinline__ void h_cell(const YeeArgs<T> &a, int i, int j, int k, bool own, T ex, T ey, T ez,
                                       T ex_y1, T ex_z1, T ey_x1, T ey_z1, T ez_x1, T ez_y1, T &hx, T &hy,
                                       T &hz) {
    T dEz_dy = ez_y1 - ez, dEy_dz = ey_z1 - ey;
    T dEx_dz = ex_z1 - ex, dEz_dx = ez_x1 - ez;
    T dEy_dx = ey_x1 - ey, dEx_dy = ex_y1 - ex;
    const int ci = canon(i, a.nx, a.per[0]), cj = canon(j, a.ny, a.per[1]), ck = canon(k, a.nz, a.per[2]);
    if (a.pml[0] | a.pml[1]) {
        int s = slab(ci, a.nx, a.pml[0], a.pml[1]);
        if (s >= 0) {
            const T *cf = a.cpml[0];
            T b = cf[3 * a.nx + ci], c = cf[4 * a.nx + ci], kk = cf[5 * a.nx + ci];
            long long q = ((long long)ck * a.ny + cj) * (a.pml[0] + a.pml[1]) + s;
            T p0 = b * a.psiHo[0][0][q] + c * dEz_dx;
            T p1 = b * a.psiHo[0][1][q] + c * dEy_dx;
            if (own) { a.psiHn[0][0][q] = p0; a.psiHn[0][1][q] = p1; }
            dEz_dx = kk * dEz_dx + p0;
            dEy_dx = kk * dEy_dx + p1;
        }
    }
    if (a.pml[2] | a.pml[3]) {
        int s = slab(cj, a.ny, a.pml[2], a.pml[3]);
        if (s >= 0) {
            const T *cf = a.cpml[1];
            T b = cf[3 * a.ny + cj], c = cf[4 * a.ny + cj], kk = cf[5 * a.ny + cj];
            long long q = ((long long)ck * (a.pml[2] + a.pml[3]) + s) * a.nx + ci;
            T p0 = b * a.psiHo[1][0][q] + c * dEz_dy;
            T p1 = b * a.psiHo[1][1][q] + c * dEx_dy;
            if (own) { a.psiHn[1][0][q] = p0; a.psiHn[1][1][q] = p1; }
            dEz_dy = kk * dEz_dy + p0;
            dEx_dy = kk * dEx_dy + p1;
        }
    }
    if (a.pml[4] | a.pml[5]) {
        int s = slab(ck, a.nz, a.pml[4], a.pml[5]);
        if (s >= 0) {
            const T *cf = a.cpml[2];
            T b = cf[3 * a.nz + ck], c = cf[4 * a.nz + ck], kk = cf[5 * a.nz + ck];
            long long q = ((long long)s * a.ny + cj) * a.nx + ci;
            T p0 = b * a.psiHo[2][0][q] + c * dEy_dz;
            T p1 = b * a.psiHo[2][1][q] + c * dEx_dz;
            if (own) { a.psiHn[2][0][q] = p0; a.psiHn[2][1][q] = p1; }
            dEy_dz = kk * dEy_dz + p0;
            dEx_dz = kk * dEx_dz + p1;
        }
    }
    hx -= a.dt * (dEz_dy - dEy_dz);
    hy -= a.dt * (dEx_dz - dEz_dx);
    hz -= a.dt * (dEy_dx - dEx_dy);
}

template <typename T>
__device__ __forceinline__ T src_value(const SrcDev &q, double t) {
    double u = (t - q.t0) / q.width;
    return (T)(q.amp * exp(-0.5 * u * u) * cos(q.omega * (t - q.t0)));
}

template <typename T>
__global__ void __launch_bounds__(TX *TY) yee_kernel(const YeeArgs<T> a) {
    __shared__ T sE[2][3][TY + 2][TX + 2];
    __shared__ T sH[3][TY + 1][TX + 1];
    __shared__ T s_src[MAXSRC];
    __shared__ int s_lo, s_hi;
    __shared__ double s_red[TX * TY / 32];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int tile = blockIdx.x;
    const int bx = tile % a.ntx, by = (tile / a.ntx) % a.nty, bz = tile / (a.ntx * a.nty);
    const int x0 = bx * TX, y0 = by * TY;
    const int k0 = bz * a.cz;
    const int k1 = min(k0 + a.cz, a.nz);
    const int i = x0 + tx, j = y0 + ty;
    const bool inb = (i < a.nx) && (j < a.ny);

    if (tid < a.nsrc) s_src[tid] = src_value<T>(a.src[tid], ((double)a.step + 0.5) * (double)a.dt);
    const int mbeg = a.tile_off ? a.tile_off[tile] : 0;
    const int mend = a.tile_off ? a.tile_off[tile + 1] : 0;
    if (tid == 0) {
        int lo = mbeg;
        while (lo < mend && a.tile_ent[lo].w <= k0 - WMAX) lo++;
        s_lo = lo;
        s_hi = lo;
    }

    // ---- prologue: H^{n+1/2}(k0-1) of the own column (z-1 neighbour of plane k0)
    T hpx, hpy, hpz;
    {
        const int km = k0 - 1;
        T ex = a.Eo[0][gi(a, i, j, km)], ey = a.Eo[1][gi(a, i, j, km)], ez = a.Eo[2][gi(a, i, j, km)];
        hpx = a.Ho[0][gi(a, i, j, km)];
        hpy = a.Ho[1][gi(a, i, j, km)];
        hpz = a.Ho[2][gi(a, i, j, km)];
        h_cell(a, i, j, km, false, ex, ey, ez, a.Eo[0][gi(a, i, j + 1, km)], a.Eo[0][gi(a, i, j, k0)],
               a.Eo[1][gi(a, i + 1, j, km)], a.Eo[1][gi(a, i, j, k0)], a.Eo[2][gi(a, i + 1, j, km)],
               a.Eo[2][gi(a, i, j + 1, km)], hpx, hpy, hpz);
    }
    // ---- stage E^n(k0) with halo
    constexpr int RW = TX + 2, RH = TY + 2, RN = RW * RH;
    for (int r = tid; r < RN; r += TX * TY) {
        int hx = r % RW, hy = r / RW;
        long long g = gi(a, x0 - 1 + hx, y0 - 1 + hy, k0);
        sE[0][0][hy][hx] = a.Eo[0][g];
        sE[0][1][hy][hx] = a.Eo[1][g];
        sE[0][2][hy][hx] = a.Eo[2][g];
    }
    double absorbed = 0.0;
    int cur = 0;
    for (int k = k0; k < k1; k++) {
        const int nxt = cur ^ 1;
        for (int r = tid; r < RN; r += TX * TY) {
            int hx = r % RW, hy = r / RW;
            long long g = gi(a, x0 - 1 + hx, y0 - 1 + hy, k + 1);
            sE[nxt][0][hy][hx] = a.Eo[0][g];
            sE[nxt][1][hy][hx] = a.Eo[1][g];
            sE[nxt][2][hy][hx] = a.Eo[2][g];
        }
        if (tid == 0) {
            int lo = s_lo, hi = s_hi;
            while (lo < mend && a.tile_ent[lo].w <= k - WMAX) lo++;
            if (hi < lo) hi = lo;
            while (hi < mend && a.tile_ent[hi].w <= k) hi++;
            s_lo = lo;
            s_hi = hi;
        }
        __syncthreads();
        // ---- H^{n+1/2}(k): own cell
        T hx, hy, hz;
        {
            const int sx = tx + 1, sy = ty + 1;
            long long g = gi(a, i, j, k);
            hx = a.Ho[0][g];
            hy = a.Ho[1][g];
            hz = a.Ho[2][g];
            h_cell(a, i, j, k, inb, sE[cur][0][sy][sx], sE[cur][1][sy][sx], sE[cur][2][sy][sx],
                   sE[cur][0][sy + 1][sx], sE[nxt][0][sy][sx], sE[cur][1][sy][sx + 1], sE[nxt][1][sy][sx],
                   sE[cur][2][sy][sx + 1], sE[cur][2][sy + 1][sx], hx, hy, hz);
            sH[0][sy][sx] = hx;
            sH[1][sy][sx] = hy;
            sH[2][sy][sx] = hz;
            if (inb) {
                store_img(a, a.Hn[0], i, j, k, hx);
                store_img(a, a.Hn[1], i, j, k, hy);
                store_img(a, a.Hn[2], i, j, k, hz);
            }
        }
        // ---- H^{n+1/2}(k): low halo row (y0-1) and column (x0-1), recomputed
        if (tid < TX + TY + 1) {
            int hxs, hys;
            if (tid < TX) { hxs = tid + 1; hys = 0; }
            else { hxs = 0; hys = tid - TX; }
            const int ii = x0 - 1 + hxs, jj = y0 - 1 + hys;
            long long g = gi(a, ii, jj, k);
            T qx = a.Ho[0][g], qy = a.Ho[1][g], qz = a.Ho[2][g];
            h_cell(a, ii, jj, k, false, sE[cur][0][hys][hxs], sE[cur][1][hys][hxs], sE[cur][2][hys][hxs],
                   sE[cur][0][hys + 1][hxs], sE[nxt][0][hys][hxs], sE[cur][1][hys][hxs + 1],
                   sE[nxt][1][hys][hxs], sE[cur][2][hys][hxs + 1], sE[cur][2][hys + 1][hxs], qx, qy, qz);
            sH[0][hys][hxs] = qx;
            sH[1][hys][hxs] = qy;
            sH[2][hys][hxs] = qz;
        }
        __syncthreads();
        // ---- E^{n+1}(k): own cell
        if (inb) {
            const int sx = tx + 1, sy = ty + 1;
            T dHz_dy = hz - sH[2][sy - 1][sx];
            T dHy_dz = hy - hpy;
            T dHx_dz = hx - hpx;
            T dHz_dx = hz - sH[2][sy][sx - 1];
            T dHy_dx = hy - sH[1][sy][sx - 1];
            T dHx_dy = hx - sH[0][sy - 1][sx];
            if (a.pml[0] | a.pml[1]) {
                int s = slab(i, a.nx, a.pml[0], a.pml[1]);
                if (s >= 0) {
                    const T *cf = a.cpml[0];
                    T b = cf[i], c = cf[a.nx + i], kk = cf[2 * a.nx + i];
                    long long q = ((long long)k * a.ny + j) * (a.pml[0] + a.pml[1]) + s;
                    T p0 = b * a.psiE[0][0][q] + c * dHz_dx;
                    T p1 = b * a.psiE[0][1][q] + c * dHy_dx;
                    a.psiE[0][0][q] = p0;
                    a.psiE[0][1][q] = p1;
                    dHz_dx = kk * dHz_dx + p0;
                    dHy_dx = kk * dHy_dx + p1;
                }
            }
            if (a.pml[2] | a.pml[3]) {
                int s = slab(j, a.ny, a.pml[2], a.pml[3]);
                if (s >= 0) {
                    const T *cf = a.cpml[1];
                    T b = cf[j], c = cf[a.ny + j], kk = cf[2 * a.ny + j];
                    long long q = ((long long)k * (a.pml[2] + a.pml[3]) + s) * a.nx + i;
                    T p0 = b * a.psiE[1][0][q] + c * dHz_dy;
                    T p1 = b * a.psiE[1][1][q] + c * dHx_dy;
                    a.psiE[1][0][q] = p0;
                    a.psiE[1][1][q] = p1;
                    dHz_dy = kk * dHz_dy + p0;
                    dHx_dy = kk * dHx_dy + p1;
                }
            }
            if (a.pml[4] | a.pml[5]) {
                int s = slab(k, a.nz, a.pml[4], a.pml[5]);
                if (s >= 0) {
                    const T *cf = a.cpml[2];
                    T b = cf[k], c = cf[a.nz + k], kk = cf[2 * a.nz + k];
                    long long q = ((long long)s * a.ny + j) * a.nx + i;
                    T p0 = b * a.psiE[2][0][q] + c * dHy_dz;
                    T p1 = b * a.psiE[2][1][q] + c * dHx_dz;
                    a.psiE[2][0][q] = p0;
                    a.psiE[2][1][q] = p1;
                    dHy_dz = kk * dHy_dz + p0;
                    dHx_dz = kk * dHx_dz + p1;
                }
            }
            T curl[3];
            curl[0] = dHz_dy - dHy_dz;
            curl[1] = dHx_dz - dHz_dx;
            curl[2] = dHy_dx - dHx_dy;
            // molecular current (fixed order of the tile list)
            T J[3] = {T(0), T(0), T(0)};
            for (int e = s_lo; e < s_hi; e++) {
                const int4 ent = a.tile_ent[e];
                const int wf = a.mol_wf[ent.x];
                const int dz = k - ent.w;
                const int dx = tx - ent.y;
                const int dy = ty - ent.z;
                if ((unsigned)dz < (unsigned)((wf >> 16) & 0xff) && (unsigned)dx < (unsigned)(wf & 0xff) &&
                    (unsigned)dy < (unsigned)((wf >> 8) & 0xff)) {
                    const T *w = a.mol_w + (long long)ent.x * NW;
                    const T *c = a.mol_c + 3ll * ent.x;
                    const T xi = w[dx], xh = w[WMAX + dx];
                    const T yi = w[2 * WMAX + dy], yh = w[3 * WMAX + dy];
                    const T zi = w[4 * WMAX + dz], zh = w[5 * WMAX + dz];
                    J[0] += c[0] * (xh * yi * zi);
                    J[1] += c[1] * (xi * yh * zi);
                    J[2] += c[2] * (xi * yi * zh);
                }
            }
            for (int q = 0; q < a.nsrc; q++) {
                const int idx3[3] = {i, j, k};
                if (idx3[a.src[q].axis] == a.src[q].index) J[a.src[q].comp] += s_src[q];
            }
            // coefficient dt/eps
            T cb = a.mat ? a.mat_cb[a.mat[((long long)k * a.ny + j) * a.nx + i]] : a.mat_cb[0];
            int midx = a.mat ? a.mat[((long long)k * a.ny + j) * a.nx + i] : 0;
            if (a.dcb && i >= a.dbox[0] && i < a.dbox[0] + a.dbox[3] && j >= a.dbox[1] &&
                j < a.dbox[1] + a.dbox[4] && k >= a.dbox[2] && k < a.dbox[2] + a.dbox[5])
                cb = a.dcb[((long long)(k - a.dbox[2]) * a.dbox[4] + (j - a.dbox[1])) * a.dbox[3] + (i - a.dbox[0])];
            bool drude = false;
            long long jq = 0;
            if (a.JD[0] && i >= a.jbox[0] && i < a.jbox[0] + a.jbox[3] && j >= a.jbox[1] &&
                j < a.jbox[1] + a.jbox[4] && k >= a.jbox[2] && k < a.jbox[2] + a.jbox[5] && a.mat_db[midx] != T(0)) {
                drude = true;
                jq = ((long long)(k - a.jbox[2]) * a.jbox[4] + (j - a.jbox[1])) * a.jbox[3] + (i - a.jbox[0]);
            }
            const int sx2 = tx + 1, sy2 = ty + 1;
            const int idx3[3] = {i, j, k};
            const long long g = gi(a, i, j, k);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const T eo = sE[cur][c][sy2][sx2];
                T jd = T(0);
                if (drude) {
                    jd = a.mat_dk[midx] * a.JD[c][jq] + a.mat_db[midx] * eo;
                    a.JD[c][jq] = jd;
                }
                bool forced = false;
#pragma unroll
                for (int b = 0; b < 3; b++)
                    if (b != c && !a.per[b] && idx3[b] == 0) forced = true;
                T en = forced ? T(0) : eo + cb * (curl[c] - J[c] - jd);
                if (drude) absorbed += (double)jd * 0.5 * ((double)eo + (double)en) * (double)a.dt;
                store_img(a, a.En[c], i, j, k, en);
            }
            (void)g;
        }
        hpx = hx;
        hpy = hy;
        hpz = hz;
        cur = nxt;
        __syncthreads();
    }
    if (a.JD[0]) {
        // fixed-order block reduction into this block's accumulator
        for (int o = 16; o > 0; o >>= 1) absorbed += __shfl_xor_sync(0xffffffffu, absorbed, o);
        if (tx == 0) s_red[ty] = absorbed;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int q = 0; q < TX * TY / 32; q++) s += s_red[q];
            a.absorbed_part[blockIdx.x] += s;
        }
    }
}

template <typename T>
cudaError_t launch_yee(const YeeArgs<T> &a, int nblocks, cudaStream_t s) {
    yee_kernel<T><<<nblocks, dim3(TX, TY), 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ field utilities

template <typename T>
__global__ void pack_kernel(const T *src, T *dst, int nx, int ny, int nz, int px, long long plane, int to_padded) {
    long long n = (long long)nx * ny * nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % nx);
        long long r = t / nx;
        int j = (int)(r % ny);
        int k = (int)(r / ny);
        long long g = (long long)(k + 1) * plane + (long long)(j + 1) * px + (i + XO);
        if (to_padded) dst[g] = src[t];
        else dst[t] = src[g];
    }
}

template <typename T>
cudaError_t launch_pack_fields(const T *src, T *dst, int nx, int ny, int nz, int px, long long plane,
                               int to_padded, cudaStream_t s) {
    long long n = (long long)nx * ny * nz;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    pack_kernel<T><<<blocks, 256, 0, s>>>(src, dst, nx, ny, nz, px, plane, to_padded);
    return cudaGetLastError();
}

// Copy periodic images into the ghost layers (after the interior was overwritten).
template <typename T>
__global__ void ghost_kernel(T *f, int nx, int ny, int nz, int px, long long plane, int p0, int p1, int p2) {
    // iterate over every padded cell in [-1,n] x [-1,n] x [-1,n] that is a ghost
    long long n = (long long)(nx + 2) * (ny + 2) * (nz + 2);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % (nx + 2)) - 1;
        long long r = t / (nx + 2);
        int j = (int)(r % (ny + 2)) - 1;
        int k = (int)(r / (ny + 2)) - 1;
        bool gx = i < 0 || i >= nx, gy = j < 0 || j >= ny, gz = k < 0 || k >= nz;
        if (!(gx || gy || gz)) continue;
        if ((gx && !p0) || (gy && !p1) || (gz && !p2)) continue;  // wall ghosts stay 0
        int si = i < 0 ? i + nx : (i >= nx ? i - nx : i);
        int sj = j < 0 ? j + ny : (j >= ny ? j - ny : j);
        int sk = k < 0 ? k + nz : (k >= nz ? k - nz : k);
        f[(long long)(k + 1) * plane + (long long)(j + 1) * px + (i + XO)] =
            f[(long long)(sk + 1) * plane + (long long)(sj + 1) * px + (si + XO)];
    }
}

template <typename T>
cudaError_t launch_refresh_ghosts(T *f, int nx, int ny, int nz, int px, long long plane, const int *per,
                                  cudaStream_t s) {
    long long n = (long long)(nx + 2) * (ny + 2) * (nz + 2);
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    ghost_kernel<T><<<blocks, 256, 0, s>>>(f, nx, ny, nz, px, plane, per[0], per[1], per[2]);
    return cudaGetLastError();
}

// Zero tangential E on the index-0 walls of non-periodic axes.
template <typename T>
__global__ void pec_kernel(T *ex, T *ey, T *ez, int nx, int ny, int nz, int px, long long plane, int p0, int p1,
                           int p2) {
    long long n = (long long)nx * ny * nz;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int i = (int)(t % nx);
        long long r = t / nx;
        int j = (int)(r % ny);
        int k = (int)(r / ny);
        long long g = (long long)(k + 1) * plane + (long long)(j + 1) * px + (i + XO);
        if ((!p1 && j == 0) || (!p2 && k == 0)) ex[g] = T(0);
        if ((!p0 && i == 0) || (!p2 && k == 0)) ey[g] = T(0);
        if ((!p0 && i == 0) || (!p1 && j == 0)) ez[g] = T(0);
    }
}

template <typename T>
cudaError_t launch_zero_pec(T *const *E, int nx, int ny, int nz, int px, long long plane, const int *per,
                            cudaStream_t s) {
    long long n = (long long)nx * ny * nz;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 65535 * 8) blocks = 65535 * 8;
    pec_kernel<T><<<blocks, 256, 0, s>>>(E[0], E[1], E[2], nx, ny, nz, px, plane, per[0], per[1], per[2]);
    return cudaGetLastError();
}

__global__ void sum_kernel(const double *src, int n, double *dst) {
    // single-thread fixed-order sum (small n: one accumulator per block of the field pass)
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < n; q++) s += src[q];
        *dst = s;
    }
}

cudaError_t launch_sum_doubles(const double *src, int n, double *dst, cudaStream_t s) {
    sum_kernel<<<1, 32, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

#define ML_INST(T)                                                                                            \
    template cudaError_t launch_yee<T>(const YeeArgs<T> &, int, cudaStream_t);                               \
    template cudaError_t launch_pack_fields<T>(const T *, T *, int, int, int, int, long long, int, cudaStream_t); \
    template cudaError_t launch_refresh_ghosts<T>(T *, int, int, int, int, long long, const int *, cudaStream_t); \
    template cudaError_t launch_zero_pec<T>(T *const *, int, int, int, int, long long, const int *, cudaStream_t);
ML_INST(float)
ML_INST(double)

}  // namespace ml
