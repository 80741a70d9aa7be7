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
//   * the dispersive poles of the pole box (Drude and Lorentz, up to four per
//     material, each its own auxiliary-differential equation; currents summed),
//   * soft current-sheet sources,
//   * the molecular current J = sum_m gamma_m mudot_m kappa_m (Eq. J_mol with
//     Eq. Polarization_mol), read from the box the current kernel wrote this step
//     (deterministic there, no atomics).
// E and H are read from one time level and written to the other, so tiles never
// race.  E^n planes are staged in shared memory (k and k+1 with halo); H^{n+1/2}
// of plane k with its low halo lives in shared memory for the E update, the own
// column's H^{n+1/2}(k-1) in registers.
#include "ml_internal.cuh"
#include "tma.cuh"

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

// Curl differences of E^n around H cell o (Eq. Maxwell b): Ek / Ek1 point at Ex of the
// staged planes k / k+1 (components BP apart), o = row * BOXW + col.
// d = {dEz/dy, dEy/dz, dEx/dz, dEz/dx, dEy/dx, dEx/dy}.
template <typename T, int BP>
__device__ __forceinline__ void e_diffs(const T *Ek, const T *Ek1, int o, T (&d)[6]) {
    const T ex = Ek[o], ey = Ek[BP + o], ez = Ek[2 * BP + o];
    d[0] = Ek[2 * BP + o + BOXW] - ez;
    d[1] = Ek1[BP + o] - ey;
    d[2] = Ek1[o] - ex;
    d[3] = Ek[2 * BP + o + 1] - ez;
    d[4] = Ek[BP + o + 1] - ey;
    d[5] = Ek[o + BOXW] - ex;
}

template <typename T>
__device__ __forceinline__ void h_finish(T dt, const T (&d)[6], T &hx, T &hy, T &hz) {
    hx -= dt * (d[0] - d[1]);
    hy -= dt * (d[2] - d[3]);
    hz -= dt * (d[4] - d[5]);
}

// CPML recursive convolution (Roden-Gedney, Taflove & Hagness Ch. 7) on one pair of
// curl terms whose derivative crosses a layer: psi' = b psi + c d, d' = kinv d + psi'.
template <typename T>
__device__ __forceinline__ void cpml_pair(T b, T c, T kinv, T &d0, T &d1, T &p0, T &p1) {
    p0 = b * p0 + c * d0;
    p1 = b * p1 + c * d1;
    d0 = kinv * d0 + p0;
    d1 = kinv * d1 + p1;
}

template <typename T>
__device__ __forceinline__ T src_value(const SrcDev &q, double t) {
    double u = (t - q.t0) / q.width;
    return (T)(q.amp * exp(-0.5 * u * u) * cos(q.omega * (t - q.t0)));
}

constexpr uint32_t WAIT_LIMIT = 2000;  // probes of up to 1 ms each before giving up

// Body of the field pass for one block.  MODE 0 is the interior form: the caller
// guarantees the tile and its halo touch no CPML layer, wall or material/source cell,
// so none of those paths is compiled in.  MODE 1 adds the CPML layers and the index-0
// walls; MODE 4 adds to those the source sheets and the per-cell coefficient dt/eps of a
// material index (from a shared-memory table); MODE 3 is the interior form with the
// source sheets and the material table, for tiles clear of the layers and walls; MODE 2
// has every path (dispersive poles, design box).  The CPML body is kept without the
// tables: their registers cost the vacuum layers' tiles time even where the tables are
// never read.  No body writes periodic ghost images: every body stores its own cells
// only, and image_kernel copies the images after the pass.
// Returns false when a plane wait gave up (the block then reported ML_ERR_TIMEOUT and
// drained its copies); uniform over the block.
template <typename T, int MODE>
__device__ __forceinline__ bool yee_body(const YeeArgs<T> &a, const TmapSet &maps, const int tile) {
    constexpr bool GEN = MODE == 1 || MODE == 2 || MODE == 4, FULL = MODE == 2;
    constexpr bool MATF = MODE == 3 || MODE == 4;  // sources and materials from the tables, no pole work
    constexpr bool MATT = MATF;                    // material table
    constexpr int S = yee_stages<T>();
    constexpr int BP = box_pad<T>();
    constexpr int SW = 6 * BP;  // elements per stage
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    T *stages = reinterpret_cast<T *>(smem_raw + 128);
    T *sHp = stages + S * SW;
    T(*sH)[TY + 1][TX + 1] = reinterpret_cast<T(*)[TY + 1][TX + 1]>(sHp);
    // Static shared arrays are sized for the bodies that use them (every body's arrays add
    // to the kernel's footprint, and a larger shared-memory carve-out leaves less L1).
    constexpr int NSRC_S = (FULL || MATF) ? MAXSRC : 1;
    __shared__ T s_src[NSRC_S];
    __shared__ double s_red[FULL ? NTHREADS / 32 : 1];
    __shared__ T sCx[GEN ? 6 : 1][GEN ? BOXW : 1];  // CPML coefficients at x = x0-4+col (bE cE kE bH cH kH)
    __shared__ T sCy[GEN ? 6 : 1][GEN ? BOXH : 1];  // at y = y0-1+row
    __shared__ T s_cb[MATT ? ML_MAX_MATERIALS : 1];  // dt / eps_inf per material (MODES 3, 4)
    // the grid's sources and flux planes (read per cell from here, not from the kernel
    // parameters: a dynamically indexed parameter array would be copied to local memory)
    __shared__ int s_sax[NSRC_S], s_sidx[NSRC_S], s_scmp[NSRC_S];
    __shared__ int s_pax[MAXPLANES], s_pidx[MAXPLANES], s_pnb[MAXPLANES], s_pnc[MAXPLANES];
    __shared__ T *s_pbuf[MAXPLANES];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int bx = tile % a.ntx, by = (tile / a.ntx) % a.nty, bz = tile / (a.ntx * a.nty);
    const int x0 = bx * TX, y0 = by * TY;
    const int k0 = a.zcut[bz];
    const int k1 = a.zcut[bz + 1];
    const int i = x0 + tx;
    const int jb = y0 + ty * RY;  // first own row; own rows jb .. jb+RY-1
    const int q0 = k0 - 1;        // first plane of the ring
    const int qlast = k1;         // last plane needed (z+1 neighbour of the last own plane)
    // bytes a stage receives: three E boxes of BOXH rows and three H boxes of BOXHH rows
    constexpr uint32_t STAGE_BYTES = 3u * BOXW * (BOXH + BOXHH) * sizeof(T);

    // block-uniform features: CPML layers this tile (with its halo) can touch, per-cell
    // material work, molecular current (periodic ghost images are written after the pass
    // by image_kernel)
    const bool fx = GEN && (a.pml[0] | a.pml[1]) && (x0 - 1 < a.pml[0] || x0 + TX > a.nx - a.pml[1]);
    const bool fy = GEN && (a.pml[2] | a.pml[3]) && (y0 - 1 < a.pml[2] || y0 + TY > a.ny - a.pml[3]);
    const bool zl = GEN && (a.pml[4] | a.pml[5]) != 0;
    const bool walls = GEN && ((!a.per[0] && x0 == 0) || (!a.per[1] && y0 == 0) || (!a.per[2] && k0 == 0));
    // per-cell material work (material table, design box, poles, sources): only tiles
    // whose own cells need it, when the grid has the per-tile flags
    const bool general = FULL && (a.tflags ? (a.tflags[tile] & 7) != 0
                                          : (a.mat != nullptr || a.dcb != nullptr || a.JD != nullptr || a.nsrc > 0));
    // MODES 3 and 4: does the tile hold a non-background material?
    const bool has_mat = MATT && a.mat != nullptr && (a.tflags ? (a.tflags[tile] & 2) != 0 : true);

    // does the tile's column meet the box of the molecular current?
    const bool has_mol = (a.Jb[0] || a.Jb[1] || a.Jb[2]) && x0 < a.jb0[0] + a.jbn[0] &&
                         x0 + TX > a.jb0[0] && y0 < a.jb0[1] + a.jbn[1] && y0 + TY > a.jb0[1] &&
                         k0 < a.jb0[2] + a.jbn[2] && k1 > a.jb0[2];
    // A tile that reads the molecular current waits for the current kernel when the
    // pass was launched as its programmatic dependent (a no-op otherwise).
    if (has_mol) pdl_wait();
    // Release the next step's molecule kernel when it is launched as this pass's
    // programmatic dependent: it stages its own state, then waits for this pass to
    // complete before it reads the field.  A tile that waited above releases it only
    // afterwards, so a release also implies that this step's molecule and current
    // kernels are complete.
    pdl_trigger();
    const T cb0 = a.mat_cb[0];
    const int col = tx + 4;
    const int ob = (ty * RY + 1) * BOXW + col;       // first own cell inside a staged box
    const int gb = (jb + 1) * a.px + (i + XO);       // first own cell inside a padded plane
    const int dxt = a.pml[0] + a.pml[1], dyt = a.pml[2] + a.pml[3];
    const bool xin = i < a.nx;
    // CPML slab coordinates of the own cells
    const int ic = canon(i, a.nx, a.per[0]);
    const int sxo = fx ? slab(ic, a.nx, a.pml[0], a.pml[1]) : -1;
    int syo[RY];
#pragma unroll
    for (int r = 0; r < RY; r++) syo[r] = fy ? slab(canon(jb + r, a.ny, a.per[1]), a.ny, a.pml[2], a.pml[3]) : -1;
    // halo cells: row y0-1 (x0..x0+TX-1) and column x0-1 (y0-1..y0+TY-1)
    const bool halo = tid < TX + TY + 1;
    const int hxs = tid < TX ? tid + 1 : 0, hys = tid < TX ? 0 : tid - TX;
    const int hic = canon(x0 - 1 + hxs, a.nx, a.per[0]), hjc = canon(y0 - 1 + hys, a.ny, a.per[1]);
    const int sxh = fx ? slab(hic, a.nx, a.pml[0], a.pml[1]) : -1;
    const int syh = fy ? slab(hjc, a.ny, a.pml[2], a.pml[3]) : -1;
    const int oh = hys * BOXW + hxs + 3;

    // (compile-time indices into the parameter arrays: indexing them by the thread
    // would make the compiler copy them to local memory)
    if (FULL || MATF)
#pragma unroll
        for (int q = 0; q < MAXSRC; q++)
            if (tid == q && q < a.nsrc) {
                s_src[q] = src_value<T>(a.src[q], ((double)a.step + 0.5) * (double)a.dt);
                s_sax[q] = a.src[q].axis;
                s_sidx[q] = a.src[q].index;
                s_scmp[q] = a.src[q].comp;
            }
#pragma unroll
    for (int p = 0; p < MAXPLANES; p++)
        if (tid == p && p < a.nplanes) {
            s_pax[p] = a.planes[p].axis;
            s_pidx[p] = a.planes[p].index;
            s_pnb[p] = a.planes[p].nb;
            s_pnc[p] = a.planes[p].nc;
            s_pbuf[p] = a.planes[p].buf;
        }
    if (MATT && tid < ML_MAX_MATERIALS) s_cb[tid] = a.mat_cb[tid];
    if (fx)
        for (int t = tid; t < 6 * BOXW; t += NTHREADS) {
            const int r = t / BOXW, cc = t % BOXW;
            sCx[r][cc] = a.cpml[0][r * a.nx + canon(x0 - 4 + cc, a.nx, a.per[0])];
        }
    if (fy)
        for (int t = tid; t < 6 * BOXH; t += NTHREADS) {
            const int r = t / BOXH, rr = t % BOXH;
            sCy[r][rr] = a.cpml[1][r * a.ny + canon(y0 - 1 + rr, a.ny, a.per[1])];
        }
    if (tid == 0) {
        for (int s = 0; s < S; s++) mbar_init(&bars[s], 1);
        fence_mbar_init();
        for (int c = 0; c < 3; c++) { prefetch_tmap(&maps.E[c]); prefetch_tmap(&maps.H[c]); }
    }
    __syncthreads();
    // does a source sheet or a flux plane cross the tile (block-uniform)?
    auto crosses = [&](int ax, int idx) {
        const int lo = ax == 0 ? x0 : (ax == 1 ? y0 : k0), hi = ax == 0 ? x0 + TX : (ax == 1 ? y0 + TY : k1);
        return idx >= lo && idx < hi;
    };
    bool has_src = false, has_pl = false;
    if (MATF)
        for (int q = 0; q < a.nsrc; q++) has_src = has_src || crosses(s_sax[q], s_sidx[q]);
    for (int p = 0; p < a.nplanes; p++) has_pl = has_pl || crosses(s_pax[p], s_pidx[p]);
    // flux planes through an own column (x- or y-normal) or crossing the chunk (z-normal,
    // checked per plane)
    static_assert(RY <= 3 && MAXPLANES <= 8, "fmask layout");
    unsigned fmask = 0;  // bits 8 + 8 r ..: the planes of own row r
    if (has_pl)
#pragma unroll
        for (int r = 0; r < RY; r++)
            for (int p = 0; p < a.nplanes; p++) {
                const int ax = s_pax[p], idx = s_pidx[p];
                if (ax == 2 ? (idx >= k0 && idx < k1) : ((ax == 0 ? i : jb + r) == idx)) fmask |= 256u << (8 * r + p);
            }
    // producer: one thread issues the six tiled loads of plane q into its stage.  The E
    // boxes start at x0 - 4 (x0 - 1 and x0 + 32 are needed) and hold rows y0 - 1 .. y0 + 8;
    // the H boxes start at x0 - 8 and end at x0 + 31 (H is needed at x0 - 1 and the own
    // columns only), so an H row is five 32-byte sectors instead of six, and hold rows
    // y0 - 1 .. y0 + 7 (no H of row y0 + 8 is read).  H of column x in a stage sits four
    // places to the right of E of column x.
    auto issue = [&](int q) {
        const int s = (q - q0) % S;
        T *st = stages + s * SW;
        mbar_expect_tx(&bars[s], STAGE_BYTES);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            tma_load_3d(st + c * BP, &maps.E[c], x0 + BOXX, y0, q + 1, &bars[s]);
            tma_load_3d(st + (3 + c) * BP, &maps.H[c], x0 + BOXX - 4, y0, q + 1, &bars[s]);
        }
    };
    int issued = q0 - 1;
    if (tid == 0)
        for (int q = q0; q <= qlast && q < q0 + S; q++) { issue(q); issued = q; }
    bool ok = true;
    auto wait_stage = [&](int s, uint32_t par) {
        if (ok && !mbar_wait_bounded(&bars[s], par, a.wait_limit)) ok = false;
    };
    auto zslab = [&](int kc) { return zl ? slab(kc, a.nz, a.pml[4], a.pml[5]) : -1; };
    // Offsets of a cell at canonical (xc, yc, kc) in the three slab stores (-1 outside
    // a layer); the stores hold fewer than 2^31 elements, so 32-bit offsets suffice,
    // computed once per cell and plane for every load and store of the plane.
    struct SlabOff { int x, y, z; };
    auto slab_off = [&](int xc, int yc, int kc, int sx, int sy, int sz) {
        SlabOff q;
        q.x = sx >= 0 ? (kc * a.ny + yc) * dxt + sx : -1;
        q.y = sy >= 0 ? (kc * dyt + sy) * a.nx + xc : -1;
        q.z = sz >= 0 ? (sz * a.ny + yc) * a.nx + xc : -1;
        return q;
    };
    // H-side CPML memory (p = {x0, x1, y0, y1, z0, z1}), old level, loaded ahead of use
    auto h_pml_load = [&](T (&p)[6], const SlabOff &q) {
        if (q.x >= 0) { p[0] = a.psiHo[0][0][q.x]; p[1] = a.psiHo[0][1][q.x]; }
        if (q.y >= 0) { p[2] = a.psiHo[1][0][q.y]; p[3] = a.psiHo[1][1][q.y]; }
        if (q.z >= 0) { p[4] = a.psiHo[2][0][q.z]; p[5] = a.psiHo[2][1][q.z]; }
    };
    // apply the recursion (coefficient column cx of sCx, row ry of sCy, plane kc) and,
    // for an own cell, store the new memory in the other time level
    auto h_pml = [&](T (&d)[6], T (&p)[6], const SlabOff &q, int kc, int cx, int ry, bool own) {
        if (q.x >= 0) {
            cpml_pair(sCx[3][cx], sCx[4][cx], sCx[5][cx], d[3], d[4], p[0], p[1]);
            if (own) { a.psiHn[0][0][q.x] = p[0]; a.psiHn[0][1][q.x] = p[1]; }
        }
        if (q.y >= 0) {
            cpml_pair(sCy[3][ry], sCy[4][ry], sCy[5][ry], d[0], d[5], p[2], p[3]);
            if (own) { a.psiHn[1][0][q.y] = p[2]; a.psiHn[1][1][q.y] = p[3]; }
        }
        if (q.z >= 0) {
            const T *cf = a.cpml[2];
            cpml_pair(cf[3 * a.nz + kc], cf[4 * a.nz + kc], cf[5 * a.nz + kc], d[1], d[2], p[4], p[5]);
            if (own) { a.psiHn[2][0][q.z] = p[4]; a.psiHn[2][1][q.z] = p[5]; }
        }
    };

    // ---- prologue: H^{n+1/2}(k0-1) of the own column (z-1 neighbour of plane k0)
    wait_stage(0, 0);
    wait_stage(1 % S, S == 1 ? 1u : 0u);
    T hpx[RY], hpy[RY];
    {
        const T *Ek = stages, *Ek1 = stages + SW;
        const int kc = canon(q0, a.nz, a.per[2]);
        const int sz = zslab(kc);
#pragma unroll
        for (int r = 0; r < RY; r++) {
            const int o = ob + r * BOXW;
            T d[6];
            e_diffs<T, BP>(Ek, Ek1, o, d);
            if (sxo >= 0 || syo[r] >= 0 || sz >= 0) {
                const int jc_ = canon(jb + r, a.ny, a.per[1]);
                const SlabOff q = slab_off(ic, jc_, kc, sxo, syo[r], sz);
                T p[6];
                h_pml_load(p, q);
                h_pml(d, p, q, kc, col, ty * RY + r + 1, false);
            }
            T hz = Ek[5 * BP + o + 4];
            hpx[r] = Ek[3 * BP + o + 4];
            hpy[r] = Ek[4 * BP + o + 4];
            h_finish(a.dt, d, hpx[r], hpy[r], hz);
        }
    }
    if (__syncthreads_or(!ok)) goto drain;
    if (tid == 0 && q0 + S <= qlast) {
        fence_proxy_async();
        issue(q0 + S);
        issued = q0 + S;
    }
    {
        // work done on the pole current, sum of J^{n+1/2} . (E^n + E^{n+1}) over the
        // thread's cells in the field precision (GB300's FP64 rate is a small fraction
        // of its FP32 rate); times dt/2 and summed in FP64 across the block
        T absorbed = T(0);
        // MODES 3 and 4: material index of the own cell, plane by plane (loaded before the wait)
        // offset of the own cell's material byte (32-bit: a grid with a material map has
        // fewer than 2^32 cells, checked when it is created)
        const unsigned nxy = (unsigned)a.nx * (unsigned)a.ny;
        unsigned mo = has_mat ? ((unsigned)k0 * (unsigned)a.ny + (unsigned)jb) * (unsigned)a.nx + (unsigned)i : 0u;
        int sc = 1 % S;               // stage of plane k (= k0 = q0 + 1)
        int sn = 2 % S;               // stage of plane k + 1
        uint32_t pn = S > 2 ? 0u : 1u;  // parity of the fill of stage sn that holds plane k + 1
        for (int k = k0; k < k1; k++) {
            const int sz = zslab(k);
            // CPML memory of this plane, loaded before the plane wait so that its
            // latency overlaps the wait and the H phase (own H side, own E side, halo H side)
            T ph[RY][6], pe[RY][6], phh[6];
            bool pown[RY];
            SlabOff qo[RY], qh;
#pragma unroll
            for (int r = 0; r < RY; r++) {
                const int j = jb + r;
                pown[r] = xin && j < a.ny && (sxo >= 0 || syo[r] >= 0 || sz >= 0);
                if (pown[r]) {
                    qo[r] = slab_off(i, j, k, sxo, syo[r], sz);
                    h_pml_load(ph[r], qo[r]);
                    if (qo[r].x >= 0) { pe[r][0] = a.psiE[0][0][qo[r].x]; pe[r][1] = a.psiE[0][1][qo[r].x]; }
                    if (qo[r].y >= 0) { pe[r][2] = a.psiE[1][0][qo[r].y]; pe[r][3] = a.psiE[1][1][qo[r].y]; }
                    if (qo[r].z >= 0) { pe[r][4] = a.psiE[2][0][qo[r].z]; pe[r][5] = a.psiE[2][1][qo[r].z]; }
                }
            }
            const bool phalo = halo && (sxh >= 0 || syh >= 0 || sz >= 0);
            if (phalo) {
                qh = slab_off(hic, hjc, k, sxh, syh, sz);
                h_pml_load(phh, qh);
            }
            int midx_l[RY];
#pragma unroll
            for (int r = 0; r < RY; r++)
                midx_l[r] = (MATT && has_mat && xin && jb + r < a.ny) ? (int)a.mat[mo + (unsigned)(r * a.nx)] : 0;
            wait_stage(sn, pn);
            const T *Ek = stages + sc * SW, *Ek1 = stages + sn * SW, *Hk = Ek + 3 * BP;
            const long long pb = (long long)(k + 1) * a.plane;
            // molecular current J^{n+1/2} of the own cells (box written by the current kernel)
            T J0[RY], J1[RY], J2[RY];
#pragma unroll
            for (int r = 0; r < RY; r++) J0[r] = J1[r] = J2[r] = T(0);
            if (has_mol) {
                const int kr = k - a.jb0[2], xr = i - a.jb0[0];
                if ((unsigned)kr < (unsigned)a.jbn[2] && (unsigned)xr < (unsigned)a.jbn[0]) {
#pragma unroll
                    for (int r = 0; r < RY; r++) {
                        const int yr = jb + r - a.jb0[1];
                        if ((unsigned)yr < (unsigned)a.jbn[1]) {
                            const long long q = ((long long)kr * a.jbn[1] + yr) * a.jbn[0] + xr;
                            if (a.Jb[0]) J0[r] = a.Jb[0][q];
                            if (a.Jb[1]) J1[r] = a.Jb[1][q];
                            if (a.Jb[2]) J2[r] = a.Jb[2][q];
                        }
                    }
                }
            }
            // ---- H^{n+1/2}(k): own cells
            T hx[RY], hy[RY], hz[RY];
#pragma unroll
            for (int r = 0; r < RY; r++) {
                const int o = ob + r * BOXW;
                const int j = jb + r;
                const bool own = xin && j < a.ny;
                hx[r] = Hk[o + 4];
                hy[r] = Hk[BP + o + 4];
                hz[r] = Hk[2 * BP + o + 4];
                T d[6];
                e_diffs<T, BP>(Ek, Ek1, o, d);
                if (pown[r]) h_pml(d, ph[r], qo[r], k, col, ty * RY + r + 1, true);
                h_finish(a.dt, d, hx[r], hy[r], hz[r]);
                const int sr = ty * RY + r + 1;
                sH[0][sr][tx + 1] = hx[r];
                sH[1][sr][tx + 1] = hy[r];
                sH[2][sr][tx + 1] = hz[r];
                if (own) {
                    // the new level is not read again in this pass: streaming
                    // (evict-first) stores leave L2 to the planes that neighbouring
                    // tiles still read as halos
                    const long long g = pb + gb + r * a.px;
                    __stcs(&a.Hn[0][g], hx[r]);
                    __stcs(&a.Hn[1][g], hy[r]);
                    __stcs(&a.Hn[2][g], hz[r]);
                }
            }
            // ---- H^{n+1/2}(k): low halo row (y0-1) and column (x0-1), recomputed
            if (halo) {
                T qx = Hk[oh + 4], qy = Hk[BP + oh + 4], qz = Hk[2 * BP + oh + 4];
                T d[6];
                e_diffs<T, BP>(Ek, Ek1, oh, d);
                if (phalo) h_pml(d, phh, qh, k, hxs + 3, hys, false);
                h_finish(a.dt, d, qx, qy, qz);
                sH[0][hys][hxs] = qx;
                sH[1][hys][hxs] = qy;
                sH[2][hys][hxs] = qz;
            }
            __syncthreads();  // publishes sH of this plane
            // ---- E^{n+1}(k): own cells
#pragma unroll
            for (int r = 0; r < RY; r++) {
                const int j = jb + r;
                if (!(xin && j < a.ny)) continue;
                const int sr = ty * RY + r + 1;
                const int o = ob + r * BOXW;
                T dHz_dy = hz[r] - sH[2][sr - 1][tx + 1];
                T dHy_dz = hy[r] - hpy[r];
                T dHx_dz = hx[r] - hpx[r];
                T dHz_dx = hz[r] - sH[2][sr][tx];
                T dHy_dx = hy[r] - sH[1][sr][tx];
                T dHx_dy = hx[r] - sH[0][sr - 1][tx + 1];
                if (pown[r]) {
                    const SlabOff &q = qo[r];
                    if (q.x >= 0) {
                        cpml_pair(sCx[0][col], sCx[1][col], sCx[2][col], dHz_dx, dHy_dx, pe[r][0], pe[r][1]);
                        a.psiE[0][0][q.x] = pe[r][0];
                        a.psiE[0][1][q.x] = pe[r][1];
                    }
                    if (q.y >= 0) {
                        cpml_pair(sCy[0][sr], sCy[1][sr], sCy[2][sr], dHz_dy, dHx_dy, pe[r][2], pe[r][3]);
                        a.psiE[1][0][q.y] = pe[r][2];
                        a.psiE[1][1][q.y] = pe[r][3];
                    }
                    if (q.z >= 0) {
                        const T *cf = a.cpml[2];
                        cpml_pair(cf[k], cf[a.nz + k], cf[2 * a.nz + k], dHy_dz, dHx_dz, pe[r][4], pe[r][5]);
                        a.psiE[2][0][q.z] = pe[r][4];
                        a.psiE[2][1][q.z] = pe[r][5];
                    }
                }
                const T curl0 = dHz_dy - dHy_dz;
                const T curl1 = dHx_dz - dHz_dx;
                const T curl2 = dHy_dx - dHx_dy;
                const T eo0 = Ek[o], eo1 = Ek[BP + o], eo2 = Ek[2 * BP + o];
                T j0 = J0[r], j1 = J1[r], j2 = J2[r];
                T en0, en1, en2;
                if (MATF) {
                    if (has_src)
                        for (int q = 0; q < a.nsrc; q++) {
                            const int ax = s_sax[q];
                            if ((ax == 0 ? i : (ax == 1 ? j : k)) == s_sidx[q]) {
                                const int cmp = s_scmp[q];
                                const T v = s_src[q];
                                j0 += cmp == 0 ? v : T(0);
                                j1 += cmp == 1 ? v : T(0);
                                j2 += cmp == 2 ? v : T(0);
                            }
                        }
                    const T cb = MATT ? s_cb[midx_l[r]] : cb0;
                    en0 = eo0 + cb * (curl0 - j0);
                    en1 = eo1 + cb * (curl1 - j1);
                    en2 = eo2 + cb * (curl2 - j2);
                } else if (!general) {
                    en0 = eo0 + cb0 * (curl0 - j0);
                    en1 = eo1 + cb0 * (curl1 - j1);
                    en2 = eo2 + cb0 * (curl2 - j2);
                } else {
                    for (int q = 0; q < a.nsrc; q++) {
                        const int ax = s_sax[q];
                        const int pos = ax == 0 ? i : (ax == 1 ? j : k);
                        if (pos == s_sidx[q]) {
                            const int cmp = s_scmp[q];
                            if (cmp == 0) j0 += s_src[q];
                            else if (cmp == 1) j1 += s_src[q];
                            else j2 += s_src[q];
                        }
                    }
                    // coefficient dt/eps (material table or design box)
                    const int midx = a.mat ? a.mat[((long long)k * a.ny + j) * a.nx + i] : 0;
                    T cb = a.mat_cb[midx];
                    if (a.dcb && i >= a.dbox[0] && i < a.dbox[0] + a.dbox[3] && j >= a.dbox[1] &&
                        j < a.dbox[1] + a.dbox[4] && k >= a.dbox[2] && k < a.dbox[2] + a.dbox[5])
                        cb = a.dcb[((long long)(k - a.dbox[2]) * a.dbox[4] + (j - a.dbox[1])) * a.dbox[3] + (i - a.dbox[0])];
                    const bool pole = a.JD && i >= a.jbox[0] && i < a.jbox[0] + a.jbox[3] && j >= a.jbox[1] &&
                                      j < a.jbox[1] + a.jbox[4] && k >= a.jbox[2] && k < a.jbox[2] + a.jbox[5];
                    // dispersive poles: each slot's ADE J^{n+1/2} = dk J^{n-1/2} + db E^n - dp P^n,
                    // then P^{n+1} = P^n + dt J^{n+1/2} (Lorentz); the currents add up
                    T jd0 = T(0), jd1 = T(0), jd2 = T(0);
                    if (pole) {
                        const long long jc = a.jcnt;
                        const long long jq =
                            ((long long)(k - a.jbox[2]) * a.jbox[4] + (j - a.jbox[1])) * a.jbox[3] + (i - a.jbox[0]);
                        for (int p = 0; p < a.npole; p++) {
                            const int mk = midx * ML_MAX_POLES + p;
                            const T db = a.mat_db[mk];
                            if (db == T(0)) break;  // a material's poles fill slots 0, 1, ...
                            const T dk = a.mat_dk[mk];
                            T *J = a.JD + 3 * p * jc + jq;
                            T q0 = dk * J[0] + db * eo0;
                            T q1 = dk * J[jc] + db * eo1;
                            T q2 = dk * J[2 * jc] + db * eo2;
                            const T dp = a.PD ? a.mat_dp[mk] : T(0);
                            if (dp != T(0)) {
                                T *P = a.PD + 3 * p * jc + jq;
                                const T p0 = P[0], p1 = P[jc], p2 = P[2 * jc];
                                q0 -= dp * p0;
                                q1 -= dp * p1;
                                q2 -= dp * p2;
                                P[0] = p0 + a.dt * q0;
                                P[jc] = p1 + a.dt * q1;
                                P[2 * jc] = p2 + a.dt * q2;
                            }
                            J[0] = q0;
                            J[jc] = q1;
                            J[2 * jc] = q2;
                            jd0 += q0;
                            jd1 += q1;
                            jd2 += q2;
                        }
                    }
                    en0 = eo0 + cb * (curl0 - j0 - jd0);
                    en1 = eo1 + cb * (curl1 - j1 - jd1);
                    en2 = eo2 + cb * (curl2 - j2 - jd2);
                    if (pole)
                        absorbed += jd0 * (eo0 + en0) + jd1 * (eo1 + en1) + jd2 * (eo2 + en2);
                }
                if (walls) {
                    // tangential E on an index-0 wall stays 0 (PEC)
                    const bool wx = !a.per[0] && i == 0, wy = !a.per[1] && j == 0, wz = !a.per[2] && k == 0;
                    if (wy || wz) en0 = T(0);
                    if (wx || wz) en1 = T(0);
                    if (wx || wy) en2 = T(0);
                }
                {
                    const long long g = pb + gb + r * a.px;
                    __stcs(&a.En[0][g], en0);
                    __stcs(&a.En[1][g], en1);
                    __stcs(&a.En[2][g], en2);
                }
                // ---- DFT flux planes through this cell: E^{n+1} and the mean of H^{n+1/2}
                // on both sides of the plane, written to the current sample slot
                for (int p = 0; p < (((fmask >> (8 + 8 * r)) & 255u) ? a.nplanes : 0); p++) {
                    if (!((fmask >> (8 + 8 * r + p)) & 1u)) continue;
                    const int ax = s_pax[p], pidx = s_pidx[p];
                    if (ax == 2 && k != pidx) continue;
                    const int per_a = ax == 0 ? a.per[0] : (ax == 1 ? a.per[1] : a.per[2]);
                    const bool zero_m = pidx == 0 && !per_a;  // H(-1) is the wall ghost (0)
                    T eb, ec, hb, hc, hbm, hcm;
                    int u, v;
                    if (ax == 2) {
                        eb = en0; ec = en1; hb = hx[r]; hc = hy[r]; hbm = hpx[r]; hcm = hpy[r]; u = i; v = j;
                    } else if (ax == 0) {
                        eb = en1; ec = en2; hb = hy[r]; hc = hz[r]; hbm = sH[1][sr][tx]; hcm = sH[2][sr][tx]; u = j; v = k;
                    } else {
                        eb = en2; ec = en0; hb = hz[r]; hc = hx[r]; hbm = sH[2][sr - 1][tx + 1]; hcm = sH[0][sr - 1][tx + 1]; u = k; v = i;
                    }
                    if (zero_m) { hbm = T(0); hcm = T(0); }
                    const int pnb = s_pnb[p];
                    T *pbuf = s_pbuf[p];
                    const long long ncell = (long long)pnb * s_pnc[p], t = (long long)v * pnb + u;
                    pbuf[t] = eb;
                    pbuf[ncell + t] = ec;
                    pbuf[2 * ncell + t] = T(0.5) * (hb + hbm);
                    pbuf[3 * ncell + t] = T(0.5) * (hc + hcm);
                }
            }
#pragma unroll
            for (int r = 0; r < RY; r++) {
                hpx[r] = hx[r];
                hpy[r] = hy[r];
            }
            if (__syncthreads_or(!ok)) goto drain;
            // the stage of plane k is free: refill it with plane k + S
            if (tid == 0 && k + S <= qlast) {
                fence_proxy_async();
                issue(k + S);
                issued = k + S;
            }
            sc = sn;
            if (++sn == S) { sn = 0; pn ^= 1u; }
            if (MATT && has_mat) mo += nxy;
        }
        if (FULL && a.JD) {
            // fixed-order block reduction into this block's accumulator
            double ab = 0.5 * (double)a.dt * (double)absorbed;
            for (int q = 16; q > 0; q >>= 1) ab += __shfl_xor_sync(0xffffffffu, ab, q);
            if (tx == 0) s_red[ty] = ab;
            __syncthreads();
            if (tid == 0) {
                double s = 0.0;
                for (int q = 0; q < NTHREADS / 32; q++) s += s_red[q];
                a.absorbed_part[tile] += s;
            }
        }
        // When the pass is a programmatic dependent, its completion must imply that of
        // the kernel before it (the next kernel's wait covers only this one).
        pdl_wait();
        return true;
    }
drain:
    // a plane never arrived: report, then wait (bounded) for the copies this block
    // issued so that none lands in shared memory after the block has exited
    if (tid == 0) {
        atomicCAS(a.status, 0, 5);
        for (int q = q0; q <= issued; q++) {
            const int s = (q - q0) % S;
            mbar_wait_bounded(&bars[s], (uint32_t)((q - q0) / S) & 1u, WAIT_LIMIT);
        }
    }
    __syncthreads();
    pdl_wait();
    return false;
}

// Per-cell work flags of a tile: bit 0 = pole box or design box, bit 1 = a
// non-background material, bit 2 = a source sheet.  Without the per-tile table every
// tile of a grid with any such feature takes the full body.
template <typename T>
__device__ __forceinline__ int tile_flags(const YeeArgs<T> &a, const int tile) {
    return a.tflags ? (int)a.tflags[tile] : ((a.mat || a.dcb || a.JD || a.nsrc) ? 1 : 0);
}

// True when the block's tile (with its one-cell halo) touches none of the CPML layers
// and walls of the field pass (the molecular current and flux-plane sampling are
// block-uniform branches of every body).  The edge of a periodic axis is interior: its
// ghost cells hold the images, written after each pass.
template <typename T>
__device__ __forceinline__ bool interior_geometry(const YeeArgs<T> &a, const int tile) {
    const int bx = tile % a.ntx, by = (tile / a.ntx) % a.nty, bz = tile / (a.ntx * a.nty);
    const int x0 = bx * TX, y0 = by * TY, k0 = a.zcut[bz], k1 = a.zcut[bz + 1];
    if ((!a.per[0] && (x0 == 0 || x0 + TX >= a.nx)) || (!a.per[1] && (y0 == 0 || y0 + TY >= a.ny)) ||
        (!a.per[2] && (k0 == 0 || k1 >= a.nz)))
        return false;
    if ((a.pml[0] && x0 - 1 < a.pml[0]) || (a.pml[1] && x0 + TX > a.nx - a.pml[1])) return false;
    if ((a.pml[2] && y0 - 1 < a.pml[2]) || (a.pml[3] && y0 + TY > a.ny - a.pml[3])) return false;
    if ((a.pml[4] && k0 - 1 < a.pml[4]) || (a.pml[5] && k1 > a.nz - a.pml[5])) return false;
    return true;
}

// 0: interior body; 1: CPML and walls (no pole or design box, material or source sheet
// in the tile); 4: CPML and walls with a material map or source sheets; 3: interior
// geometry with a material map or source sheets; 2: every path (poles, design box).
template <typename T>
__device__ __forceinline__ int block_mode(const YeeArgs<T> &a, const int tile) {
    const int fl = tile_flags(a, tile);
    if (interior_geometry(a, tile)) {
        if (fl == 0) return 0;
        if ((fl & 1) == 0) return 3;
        return 2;
    }
    return (fl & 1) != 0 ? 2 : (fl != 0 ? 4 : 1);
}

// Body of a tile in a kernel compiled with body set B.  The host picks the set from the
// bodies of all of the grid's tiles: with YEE_BODIES_VACUUM every tile takes body 0 or 1;
// with YEE_BODIES_TABLES body 0, 3 or 4 (a CPML tile without material or source takes
// body 4, which then reads the background entry of the table).
template <typename T, int B = YEE_BODIES_ALL>
__device__ __forceinline__ bool yee_dispatch(const YeeArgs<T> &a, const TmapSet &maps, const int tile) {
    const int mode = block_mode(a, tile);
    if (mode == 0) return yee_body<T, 0>(a, maps, tile);
    if (B == YEE_BODIES_VACUUM) return yee_body<T, 1>(a, maps, tile);
    if (B == YEE_BODIES_TABLES) {
        if (mode == 3) return yee_body<T, 3>(a, maps, tile);
        return yee_body<T, 4>(a, maps, tile);
    }
    if (mode == 1) return yee_body<T, 1>(a, maps, tile);
    if (mode == 3) return yee_body<T, 3>(a, maps, tile);
    if (mode == 4) return yee_body<T, 4>(a, maps, tile);
    return yee_body<T, 2>(a, maps, tile);
}

template <typename T, int B>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? 4 : 1) yee_kernel(const YeeArgs<T> a,
                                                                           const __grid_constant__ TmapSet maps) {
    const int tile = a.blist ? a.blist[blockIdx.x] : (int)blockIdx.x;
    yee_dispatch<T, B>(a, maps, tile);
}

// Batched field pass: one persistent launch for the tiles of many grids.  Each block
// walks the (instance, tile) work list; per item it copies the instance's arguments
// into shared memory, turns them to the time level, step and DFT ring slot of this
// step, and runs the same body as the single-grid kernel.
template <typename T, int B>
__global__ void __launch_bounds__(NTHREADS, sizeof(T) == 4 ? 3 : 1) yee_batch_kernel(const YeeBatch<T> b) {
    __shared__ __align__(16) YeeArgs<T> sa;
    __shared__ const TmapSet *smaps;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    const int tid = threadIdx.y * TX + threadIdx.x;
    constexpr int NW = (int)(sizeof(YeeArgs<T>) / sizeof(int));
    static_assert(sizeof(YeeArgs<T>) % sizeof(int) == 0, "argument block copied as words");
    for (int w = blockIdx.x; w < b.nwork; w += gridDim.x) {
        const int2 wk = b.work[w];
        __syncthreads();  // the previous item is done with sa and the barriers
        if (w != (int)blockIdx.x && tid == 0)
            for (int q = 0; q < yee_stages<T>(); q++) mbar_inval(&bars[q]);
        const int *src = reinterpret_cast<const int *>(b.args + wk.x);
        int *dst = reinterpret_cast<int *>(&sa);
        for (int q = tid; q < NW; q += NTHREADS) dst[q] = src[q];
        __syncthreads();
        if (tid == 0) {
            const int lev = (b.lev0[wk.x] + b.s) & 1;
            if (lev) {
                for (int c = 0; c < 3; c++) {
                    const T *e = sa.Eo[c], *h = sa.Ho[c];
                    sa.Eo[c] = sa.En[c];
                    sa.Ho[c] = sa.Hn[c];
                    sa.En[c] = const_cast<T *>(e);
                    sa.Hn[c] = const_cast<T *>(h);
                    for (int q = 0; q < 2; q++) {
                        const T *p = sa.psiHo[c][q];
                        sa.psiHo[c][q] = sa.psiHn[c][q];
                        sa.psiHn[c][q] = const_cast<T *>(p);
                    }
                }
            }
            sa.step += *b.boff + b.s;
            for (int p = 0; p < sa.nplanes; p++)
                sa.planes[p].buf += (size_t)b.slot * 4 * sa.planes[p].nb * sa.planes[p].nc;
            smaps = b.maps + 2 * wk.x + lev;
        }
        __syncthreads();
        const bool ok = yee_dispatch<T, B>(sa, *smaps, wk.y);
        // a wait that gave up may leave copies in flight: stop reusing this block
        if (!ok) return;
    }
}

template <typename T>
cudaError_t launch_yee_batch(const YeeBatch<T> &b, int grid, cudaStream_t s, bool pdl) {
    static bool configured[3] = {};
    const size_t smem = yee_smem_bytes<T>();
    const int bs = b.bodies == YEE_BODIES_VACUUM || b.bodies == YEE_BODIES_TABLES ? b.bodies : YEE_BODIES_ALL;
    void (*kern)(const YeeBatch<T>) = bs == YEE_BODIES_VACUUM   ? yee_batch_kernel<T, YEE_BODIES_VACUUM>
                                      : bs == YEE_BODIES_TABLES ? yee_batch_kernel<T, YEE_BODIES_TABLES>
                                                                : yee_batch_kernel<T, YEE_BODIES_ALL>;
    if (!configured[bs]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[bs] = true;
    }
    if (b.nwork == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TX, NTY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, b);
}

template <typename T>
cudaError_t launch_yee(const YeeArgs<T> &a, const TmapSet &maps, int nblocks, cudaStream_t s, bool pdl) {
    static bool configured[3] = {};
    const size_t smem = yee_smem_bytes<T>();
    const int b = a.bodies == YEE_BODIES_VACUUM || a.bodies == YEE_BODIES_TABLES ? a.bodies : YEE_BODIES_ALL;
    void (*kern)(const YeeArgs<T>, const TmapSet) = b == YEE_BODIES_VACUUM   ? yee_kernel<T, YEE_BODIES_VACUUM>
                                                    : b == YEE_BODIES_TABLES ? yee_kernel<T, YEE_BODIES_TABLES>
                                                                             : yee_kernel<T, YEE_BODIES_ALL>;
    if (!configured[b]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[b] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(TX, NTY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, maps);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// The body each tile of the field pass takes (block_mode), one byte per tile: the host
// orders the pass's blocks by it once, when the grid is created.
template <typename T>
__global__ void tile_modes_kernel(const YeeArgs<T> a, int ntiles, uint8_t *out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) out[t] = (uint8_t)block_mode(a, t);
}

template <typename T>
cudaError_t launch_tile_modes(const YeeArgs<T> &a, int ntiles, uint8_t *out, cudaStream_t s) {
    if (ntiles <= 0) return cudaSuccess;
    tile_modes_kernel<T><<<(ntiles + 255) / 256, 256, 0, s>>>(a, ntiles, out);
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
    template cudaError_t launch_yee<T>(const YeeArgs<T> &, const TmapSet &, int, cudaStream_t, bool);                         \
    template cudaError_t launch_yee_batch<T>(const YeeBatch<T> &, int, cudaStream_t, bool);                                  \
    template cudaError_t launch_tile_modes<T>(const YeeArgs<T> &, int, uint8_t *, cudaStream_t);                              \
    template cudaError_t launch_pack_fields<T>(const T *, T *, int, int, int, int, long long, int, cudaStream_t); \
    template cudaError_t launch_refresh_ghosts<T>(T *, int, int, int, int, long long, const int *, cudaStream_t); \
    template cudaError_t launch_zero_pec<T>(T *const *, int, int, int, int, long long, const int *, cudaStream_t);
ML_INST(float)
ML_INST(double)

}  // namespace ml
