// Internal declarations of libmaxlink (not part of the ABI).
//
// Device layout of a grid (HBM):
//   * six field arrays per time level, E and H double-buffered (ping-pong), each
//     padded with one ghost layer on every side: element (i,j,k), i in [-1, nx],
//     lives at (k+1)*plane + (j+1)*px + (i+XO).  Interior rows start 128-byte
//     aligned (XO = 32 elements, px a multiple of 32), so every warp-wide row
//     access covers whole cache lines and no partially written sector is left for
//     another block to complete.  Ghosts of non-periodic axes stay 0 (PEC wall); ghosts of
//     periodic axes are written by the owner of the mirrored cell in the same pass.
//   * CPML memory variables only inside the layers: per axis a slab of
//     (pml_lo + pml_hi) cells along a, two H-side components (double-buffered,
//     because neighbouring tiles recompute halo H from them) and two E-side
//     components (updated in place by the owning cell).
//   * per-cell uint8 material index, a continuous-eps design box, a pole box (pole
//     currents and, for Lorentz poles, polarisations per pole slot).
//   * molecule tables (SoA), per-molecule separable kernel weights, and the
//     per-block entry lists of the current box (each molecule window meeting a
//     block, in a fixed order) that make the current scatter deterministic.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "maxlink.h"

#include <string>

namespace ml {

// Message returned by ml_last_error on the calling thread.
void set_last_error(const std::string &msg);

constexpr int TX = 32;      // tile width in x (one warp)
constexpr int TY = 8;       // tile rows in y
constexpr int RY = 1;       // rows per thread (threads per block: TX x TY/RY)
constexpr int NTY = TY / RY;
constexpr int NTHREADS = TX * NTY;
constexpr int XO = 32;      // x offset of the interior in a padded row (rows start 128-byte aligned)
constexpr int WMAX = 16;    // max kernel window per axis (2 ceil(3 sigma) + 2)
constexpr int NW = 6 * WMAX;  // weights per molecule: [axis][stagger][WMAX]
constexpr int MAXLEV = 8;
constexpr int MAXSRC = 4;
constexpr int MAXPLANES = 8;
#define ML_MAX_FREQS_DEV 64
constexpr int DFT_KMAX = 64;  // samples buffered per plane before a fold

struct SrcDev {
    int axis, index, comp;
    double amp, omega, width, t0;
};

template <typename T>
struct cx {
    T re, im;
};

// ------------------------------------------------------------------ field pass
// A DFT flux plane sampled by the field pass: the two tangential E and the two
// tangential H (averaged over the half cells on both sides) of every plane cell
// are written to buf[4][nc*nb] (the current ring slot).
template <typename T>
struct PlaneDev {
    int axis, index, nb, nc;
    T *buf;
};

// Body sets of the field-pass kernel: a grid takes the smallest set that covers every
// tile's body (block_mode in yee.cu).
constexpr int YEE_BODIES_VACUUM = 0;  // interior and CPML bodies
constexpr int YEE_BODIES_TABLES = 1;  // interior, interior with tables, CPML with tables
constexpr int YEE_BODIES_ALL = 2;     // every body

template <typename T>
struct YeeArgs {
    int nx, ny, nz, px, py;
    int bodies;                 // YEE_BODIES_*: which kernel the host launches
    long long plane;
    int per[3];
    int pml[6];
    int ntx, nty, nchunk, cz;   // cz: longest chunk
    const int *blist;           // blocks of this launch (tile indices), or null for all
    const uint8_t *tflags;      // per tile: bit 0 = the pole box or the design box meets its own
                                //   cells, bit 1 = a non-background material, bit 2 = a source plane
    const int *zcut;            // chunk c covers planes [zcut[c], zcut[c+1])
    T dt;
    const T *Eo[3];
    const T *Ho[3];
    T *En[3];
    T *Hn[3];
    // CPML coefficients per axis: 6 rows of n (bE cE kE bH cH kH)
    const T *cpml[3];
    // CPML memory: per axis, H side [2] old/new, E side [2] in place
    const T *psiHo[3][2];
    T *psiHn[3][2];
    T *psiE[3][2];
    // materials
    const uint8_t *mat;   // (nz,ny,nx) or null
    const T *mat_cb;      // dt / eps_inf per material
    const T *mat_dk;      // pole recursion factor [material * ML_MAX_POLES + slot]
    const T *mat_db;      // pole drive factor, same layout (0 = no pole in the slot)
    const T *mat_dp;      // pole restoring factor, same layout (0 = Drude)
    int dbox[6];
    const T *dcb;         // dt / eps per design-box cell
    int jbox[6];
    int npole;            // pole slots in use (0: no poles)
    long long jcnt;       // cells of the pole box
    T *JD;                // pole currents [slot][component][jcnt] over the pole box (null: none)
    T *PD;                // pole polarisations, same layout (null: no Lorentz pole)
    double *absorbed_part;  // one accumulator per block
    // molecular current on its box (written by the current kernel this step)
    int jb0[3], jbn[3];     // box origin and extent in cells
    const T *Jb[3];         // per component, null if no molecule has a dipole along it
    int nsrc;
    SrcDev src[MAXSRC];
    int nplanes;
    PlaneDev<T> planes[MAXPLANES];
    long long step;
    int *status;
    uint32_t wait_limit;  // probes of a plane wait before it gives up (ML_ERR_TIMEOUT)
};

// TMA descriptors of the six arrays of the time level the field pass reads.
struct TmapSet {
    CUtensorMap E[3];
    CUtensorMap H[3];
};

constexpr int BOXW = TX + 8;   // TMA box: x0-4 .. x0+TX+3 (16-byte aligned start)
constexpr int BOXX = XO - 4;   // padded x index of the box start minus x0
constexpr int BOXH = TY + 2;   // rows y0-1 .. y0+TY (E)
constexpr int BOXHH = TY + 1;  // rows y0-1 .. y0+TY-1 (H: the curl of E needs E at y0+TY, never H)
template <typename T> constexpr int yee_stages() { return sizeof(T) == 4 ? 4 : 3; }
template <typename T> constexpr int box_pad() { return (int)(((BOXW * BOXH * sizeof(T) + 127) / 128) * 128 / sizeof(T)); }
template <typename T> constexpr size_t yee_smem_bytes() {
    return 128 + (size_t)yee_stages<T>() * 6 * box_pad<T>() * sizeof(T) + 3 * (TY + 1) * (TX + 1) * sizeof(T) + 64;
}

// ------------------------------------------------------------------ current
constexpr int JX = 32, JY = 8, JZ = 8;  // cells per block of the current kernel

template <typename T>
struct CurArgs {
    int nblocks, nbx, nby;
    int bn[3];           // box extent in cells
    const int *off;      // CSR: entries of block b are ent[off[b] .. off[b+1])
    const int4 *ent;     // (molecule, window start - block origin along x, y, z)
    const unsigned char *emask;  // per entry: bit q set when its x window meets columns 4q .. 4q+3
    const int *wf;       // per molecule: window length along x, y, z (8 bits each)
    const T *w;          // (M, NW) 1D kernel weights per axis and stagger (zero past the window)
    const T *c;          // (M, 3) gamma * mudot of this step
    int cmask;           // components with a dipole
    T *J[3];             // box arrays (nz, ny, nx of the box)
};

// Gather partials: for every (box block, entry) the field sum of the entry's kernel
// window inside the block, per component; the molecule kernel adds a molecule's
// partials in list order.
template <typename T>
struct GathArgs {
    int nblocks, nbx, nby;
    int bn[3];           // box extent in cells
    int b0[3];           // box origin in grid cells
    int px;              // padded field layout
    long long plane;
    const int *off;
    const int4 *ent;
    const int *wf;       // per molecule: window length along x, y, z (8 bits each)
    const T *w;          // (M, NW) 1D kernel weights per axis and stagger
    const int *cmask;    // per molecule
    int gcmask;          // components staged
    const T *E[3];       // E^n (padded)
    T *part;             // (entries, 3)
};

// ------------------------------------------------------------------ molecules
template <typename T>
struct MolArgs {
    int nmol;
    T dt;
    int nx, ny, nz, px;
    long long plane;
    int per[3];
    const T *E[3];
    const int *nlev;
    const long long *off;
    const int *kind;
    const int *nsub;
    const int *cmask;      // bit c set: dipole has a nonzero component along c
    const T *gamma;
    const T *decay;
    const T *dephase;
    const cx<T> *H0;
    const cx<T> *mu;       // 3 pools back to back
    long long pool;
    cx<T> *rho;
    T *Et;
    T *mudot;
    T *c;
    double *energy;
    int *status;
    const int *win;        // per molecule: canonical window start along x, y, z
    const int *wf;         // per molecule: window length along x, y, z (8 bits each)
    const T *w;            // (M, NW) 1D kernel weights per axis and stagger
    int two_level;         // every molecule has two levels, at pool offset 4 m
    int exact_only;        // (uniform-field solvers) every molecule takes the exact 2x2 step
    int mu_zero;           // (uniform-field solvers) bit c set: every molecule's mu_c is zero and is not loaded
    double *pop_sink;      // populations of the new state, device address of page-locked host memory
    long long pop_slot;    // row block of this step in the sink: (step mod ring) * nmol * MAXLEV
    const T *Eu;           // uniform-field source: the field before gamma_m (3 values, field type)
    T *gmu;                // uniform-field source: gamma_m <mu> of the new state (M, 3)
    double *dpart;         // single-mode cavity, two-level molecules: per-block sums of gamma_m <mu_x,y> (2 each)
    // single-mode cavity, two-level molecules: the launch's last block advances the mode
    double *mode;          // q_x q_y p_x p_y d_x d_y Eu_x Eu_y Eu_z (FP64)
    float *euf;            // Eu in FP32 for FP32 molecules, else null
    unsigned *ticket;      // blocks of the launch that have written their partial
    double wc, eps, mdt;   // mode frequency, coupling, time step
    // uniform-field source with laser = 1: the prescribed plane wave of Eq. E_analytical
    // instead of Eu, E~_m = gamma_m E0 pol env(u) cos(k u + phase), u = z_m - xi0 - t,
    // t = (run's first step + lstep) dt, env(u) = cos^2(pi u / 2W) for |u| < W
    int laser;
    int lstep;
    const double *zpos;     // FP64 fields: z_m
    const long long *lbase; // FP64 fields: the run's first step
    double ldt, lxi0;       // FP64 fields
    const float2 *lzr;      // FP32 fields: z_m - xi0 as a float pair (hi, lo = the FP64 remainder)
    const float2 *ltt;      // FP32 fields: t of each launch of the run as a float pair
    T lk, lphase, lW, lE0, lpol[3];
    // packed form (grids with multilevel molecules): molecules sorted by (kind, level
    // count, substeps, window position) in `order`; item i covers order[x .. x+y) with
    // level count z and w = kind | nsub << 4, one item per warp
    const int *order;
    const int4 *items;
    int nitems;
};
// Molecules per warp of the packed molecule kernel for n levels: a molecule's n(n+1)/2
// upper-triangle elements go to a group of G lanes, G the next power of two (64 for
// n = 8: two elements per lane).
__host__ __device__ constexpr int pack_group(int n) {
    return n * (n + 1) / 2 <= 4 ? 4 : (n * (n + 1) / 2 <= 8 ? 8 : (n * (n + 1) / 2 <= 16 ? 16 : (n * (n + 1) / 2 <= 32 ? 32 : 64)));
}
__host__ __device__ constexpr int pack_per_warp(int n) { return pack_group(n) <= 32 ? 32 / pack_group(n) : 1; }
constexpr int MU_THREADS_HOST = 256;  // molecules per block of the thread-per-molecule uniform-field kernel

// ------------------------------------------------------------------ DFT planes
template <typename T>
struct PlaneArgs {
    int axis, index, nb, nc;   // (a,b,c) cyclic; sample grid nb x nc (b fastest)
    int px;
    long long plane;
    int per_a, n_a;
    const T *E[3];
    const T *H[3];
    T *buf;                    // [K][4][nc*nb]
    int slot;
};

// ------------------------------------------------------------------ batches
// Many independent grids advanced by the same launches: per-instance arguments live in
// device arrays and each launch walks a list of (instance, block) work items.  A
// sequence of steps is indexed by s (baked into the launch) plus a device step counter
// (boff) that a tick kernel advances, so that a captured sequence can be replayed.
template <typename T>
struct YeeBatch {
    const YeeArgs<T> *args;   // per instance, for level 0 (reads F[0], writes F[1]), step = base
    const TmapSet *maps;      // per instance, two: level 0 and level 1
    const int *lev0;          // level each instance reads at s = 0
    const int2 *work;         // (instance, tile)
    int nwork;
    const long long *boff;
    int s;                    // step within the sequence
    int slot;                 // DFT ring slot of this step
    int bodies;               // YEE_BODIES_* covering every instance's tiles
};
template <typename T>
struct GathBatch {
    const GathArgs<T> *args;  // per instance, two: E of level 0 and of level 1
    const int *lev0;
    const int2 *work;         // (instance, box block)
    int s;
};
template <typename T>
struct CurBatch {
    const CurArgs<T> *args;
    const int2 *work;         // (instance, box block)
};
template <typename T>
struct MolBatch {
    const MolArgs<T> *args;   // per instance, two: E of level 0 and of level 1
    const int *lev0;
    const int2 *work;         // (instance, first molecule of the block)
    int s;
    int two_level;            // every instance's molecules are all two-level
};
template <typename T>
struct FoldDesc {
    const T *buf;
    int ncell, nfreq;
    const double *omega;
    const T *ph;              // the plane's table of e^{i w s dt}
    long long step_base;
    double2 *acc;
};
template <typename T>
struct FoldBatch {
    const FoldDesc<T> *desc;
    const int2 *work;         // (descriptor, chunk of 256 entries)
    int nsamp;
    const long long *boff;
    int s_first;
    double dt;
};

// launchers (explicit instantiations for float and double live in the .cu files)
template <typename T> cudaError_t launch_yee_batch(const YeeBatch<T> &b, int grid, cudaStream_t s, bool pdl = false);
template <typename T> cudaError_t launch_gather_batch(const GathBatch<T> &b, int nwork, cudaStream_t s);
template <typename T> cudaError_t launch_current_batch(const CurBatch<T> &b, int nwork, cudaStream_t s,
                                                       bool pdl = false);
template <typename T> cudaError_t launch_molecules_batch(const MolBatch<T> &b, int nwork, cudaStream_t s);
template <typename T> cudaError_t launch_fold_batch(const FoldBatch<T> &b, int nwork, cudaStream_t s);
cudaError_t launch_tick(long long *c, int add, cudaStream_t s);
// pdl: launch with programmatic stream serialisation, so that blocks that do not read
// the molecular current may start while the current kernel still runs.
template <typename T> cudaError_t launch_yee(const YeeArgs<T> &a, const TmapSet &maps, int nblocks, cudaStream_t s,
                                             bool pdl = false);
// Periodic ghost images of the six field arrays of one time level: every ghost cell on
// a face of a periodic axis takes the value of its image inside the grid (wall ghosts
// stay 0).  Run after each field pass of a grid with a periodic axis.
template <typename T>
struct ImgArgs {
    T *f[6];
    int nx, ny, nz, px;
    long long plane;
    int per[3];
};
template <typename T> cudaError_t launch_images(const ImgArgs<T> &a, cudaStream_t s);
// the field-pass body of every tile (0..4, see block_mode in yee.cu), one byte per tile
template <typename T> cudaError_t launch_tile_modes(const YeeArgs<T> &a, int ntiles, uint8_t *out, cudaStream_t s);
template <typename T> cudaError_t launch_molecules(const MolArgs<T> &a, cudaStream_t s, bool pdl = false);
template <typename T> cudaError_t launch_molecules_packed(const MolArgs<T> &a, cudaStream_t s, bool pdl = false);
template <typename T> cudaError_t launch_molecules_uniform(const MolArgs<T> &a, cudaStream_t s);
// single-mode cavity with two-level molecules: the molecule step and the mode step in one launch
template <typename T> cudaError_t launch_molecules_cavity(const MolArgs<T> &a, cudaStream_t s);
constexpr int CAV_GRID = 3 * 152;  // blocks of that launch at most: one wave of three per SM on 152 SMs

// One velocity-Verlet step of the single-mode cavity (Sec. II normal modes, single-mode
// limit) given the new dipole sums d = sum_m gamma_m <mu_x,y>; writes the next field
// Eu = -(eps q + eps^2 / wc^2 d), and its FP32 copy when euf is set.
__device__ inline void cavity_advance_mode(double *mode, float *euf, const double (&d)[2], double wc, double eps,
                                           double dt) {
    for (int l = 0; l < 2; l++) {
        const double q = mode[l], p = mode[2 + l], d0 = mode[4 + l];
        const double ph = p + 0.5 * dt * (-wc * wc * q - eps * d0);
        const double qn = q + dt * ph;
        const double pn = ph + 0.5 * dt * (-wc * wc * qn - eps * d[l]);
        mode[l] = qn;
        mode[2 + l] = pn;
        mode[4 + l] = d[l];
        mode[6 + l] = -(eps * qn + eps * eps / (wc * wc) * d[l]);
    }
    mode[8] = 0.0;
    if (euf)
        for (int l = 0; l < 3; l++) euf[l] = (float)mode[6 + l];
}
template <typename T> cudaError_t launch_current(const CurArgs<T> &a, cudaStream_t s, bool pdl = false);
template <typename T> cudaError_t launch_gather(const GathArgs<T> &a, cudaStream_t s);
template <typename T> cudaError_t launch_weights(int nmol, const double *pos, const double *sigma,
                                                 const int *win, const int *wf, const int *wraw,
                                                 const int *dims, const int *per, T *w, cudaStream_t s);
template <typename T> cudaError_t launch_dft_sample(const PlaneArgs<T> &a, cudaStream_t s);
template <typename T> cudaError_t launch_dft_fold(const T *buf, int nsamp, int ncell, int nfreq,
                                                  const double *omega, const T *ph, long long step0, double dt,
                                                  double2 *acc, cudaStream_t s);
template <typename T> cudaError_t launch_dft_phases(const double *omega, int nfreq, double dt, T *ph, cudaStream_t s);
constexpr int FLUX_NB = 64;  // blocks per frequency of the flux reduction (a power of two)
cudaError_t launch_flux_reduce(const double2 *acc, int ncell, int nfreq, double *part, double *out, cudaStream_t s);
template <typename T> cudaError_t launch_pack_fields(const T *src, T *dst, int nx, int ny, int nz, int px,
                                                     long long plane, int to_padded, cudaStream_t s);
template <typename T> cudaError_t launch_refresh_ghosts(T *f, int nx, int ny, int nz, int px, long long plane,
                                                        const int *per, cudaStream_t s);
template <typename T> cudaError_t launch_zero_pec(T *const *E, int nx, int ny, int nz, int px, long long plane,
                                                  const int *per, cudaStream_t s);
template <typename T> cudaError_t launch_mol_export(int what, int nmol, const int *nlev, const long long *off,
                                                    const cx<T> *rho, const T *Et, const T *mudot,
                                                    const double *energy, long long pool, double *dst,
                                                    cudaStream_t s);
cudaError_t launch_sum_doubles(const double *src, int n, double *dst, cudaStream_t s);

}  // namespace ml
