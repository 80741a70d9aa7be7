// Host side of libmaxlink: the C ABI of include/maxlink.h.
//
// Owns the device state of a grid, validates arguments, lays out the padded
// fields, builds the CPML and material coefficient tables, bins molecules into
// per-tile lists, and enqueues the per-step kernels:
//   K2 molecules (gather E^n, rho step, mudot)  ->  K1 fused field pass (H, E)
//   ->  K4 plane sampling (every step) / fold (every DFT_KMAX steps).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "grid.cuh"

using namespace ml;

namespace {
thread_local std::string g_err;
}  // namespace


namespace {

// zeroed device memory from the process allocator, owned by `list`
ml_status dalloc(std::vector<DevBuf> &list, void **p, size_t bytes) { return dev_alloc(list, p, bytes); }

#define AL(list, ptr, bytes)                                                \
    do {                                                                    \
        ml_status s_ = dalloc(list, (void **)&(ptr), (bytes));              \
        if (s_ != ML_OK) return s_;                                         \
    } while (0)

template <typename T>
ml_status upload_as(std::vector<DevBuf> &list, void **dst, const std::vector<double> &v) {
    std::vector<T> t(v.begin(), v.end());
    AL(list, *dst, t.size() * sizeof(T));
    if (!t.empty()) CK(cudaMemcpy(*dst, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ML_OK;
}

ml_status upload_reals(ml_grid *g, std::vector<DevBuf> &list, void **dst, const std::vector<double> &v) {
    return g->prec ? upload_as<double>(list, dst, v) : upload_as<float>(list, dst, v);
}

template <typename V>
ml_status upload_raw(std::vector<DevBuf> &list, V **dst, const std::vector<V> &v) {
    AL(list, *dst, v.size() * sizeof(V));
    if (!v.empty()) CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    return ML_OK;
}

int dim(const ml_grid *g, int a) { return a == 0 ? g->nx : (a == 1 ? g->ny : g->nz); }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA descriptor of one padded field array: 3D (px, py, nz+2), box BOXW x rows x 1.
ml_status make_tmap(const ml_grid *g, void *base, int rows, CUtensorMap *out) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
            return fail(ML_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        fn = (EncodeTiledFn)p;
    }
    cuuint64_t dims[3] = {(cuuint64_t)g->px, (cuuint64_t)g->py, (cuuint64_t)(g->nz + 2)};
    cuuint64_t strides[2] = {(cuuint64_t)g->px * g->esz, (cuuint64_t)g->plane * g->esz};
    cuuint32_t box[3] = {(cuuint32_t)BOXW, (cuuint32_t)rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(out, g->prec ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims,
                    strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ML_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    return ML_OK;
}

// Roden-Gedney CPML coefficients (Taflove & Hagness Ch. 7) at position x along axis a.
void cpml_coeff(const ml_grid *g, int a, double x, double &b, double &c, double &ik) {
    int n = dim(g, a), dl = g->pml[2 * a], dh = g->pml[2 * a + 1];
    double u = 0.0;
    if (dl > 0 && x < dl) u = (dl - x) / dl;
    else if (dh > 0 && x > n - dh) u = (x - (n - dh)) / dh;
    if (u <= 0.0) { b = 0.0; c = 0.0; ik = 1.0; return; }
    double sg = g->smax * std::pow(u, g->pml_m);
    double kp = 1.0 + (g->kmax - 1.0) * std::pow(u, g->pml_m);
    double al = g->amax * (1.0 - u);
    b = std::exp(-(sg / kp + al) * g->dt);
    c = sg > 0 ? sg / (sg * kp + kp * kp * al) * (b - 1.0) : 0.0;
    ik = 1.0 / kp;
}

}  // namespace

// Definitions below take C linkage from their declarations in maxlink.h.

const char *ml_last_error(void) { return g_err.c_str(); }

// Lets entry points defined in other files report through ml_last_error.
void ml::set_last_error(const std::string &msg) { g_err = msg; }

const char *ml_version(void) { return "maxlink-gb300 0.3 (sm_103a)"; }

ml_status ml_grid_destroy(ml_grid *g) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    cudaDeviceSynchronize();
    for (auto &x : g->timed) { g->ev_free.push_back(x.a); g->ev_free.push_back(x.b); }
    for (cudaEvent_t e : g->ev_free) cudaEventDestroy(e);
    if (g->side) cudaStreamDestroy(g->side);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->ev_box) cudaEventDestroy(g->ev_box);
    dev_free_all(g->mol_allocs);
    dev_free_all(g->allocs);
    delete g;
    return ML_OK;
}

ml_status ml_grid_create(const ml_grid_desc *d, void *stream, ml_grid **out) {
    (void)stream;
    if (!d || !out) return fail(ML_ERR_INVALID_ARG, "null descriptor or output");
    *out = nullptr;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(ML_ERR_INVALID_ARG, "grid dimensions must be >= 1");
    if ((long long)d->nx * d->ny * d->nz > (1ll << 34)) return fail(ML_ERR_INVALID_ARG, "grid too large");
    if (!(d->courant > 0.0 && d->courant <= 1.0)) return fail(ML_ERR_INVALID_ARG, "courant must be in (0, 1]");
    if (d->precision != ML_F32 && d->precision != ML_F64) return fail(ML_ERR_INVALID_ARG, "precision must be ML_F32 or ML_F64");
    const int dims[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; a++) {
        if (d->periodic[a] && (d->pml[2 * a] || d->pml[2 * a + 1]))
            return fail(ML_ERR_INVALID_ARG, "CPML on a periodic axis");
        if (d->pml[2 * a] < 0 || d->pml[2 * a + 1] < 0 || d->pml[2 * a] + d->pml[2 * a + 1] > dims[a])
            return fail(ML_ERR_INVALID_ARG, "CPML thickness out of range");
    }
    if (d->n_materials < 1 || d->n_materials > ML_MAX_MATERIALS || !d->materials)
        return fail(ML_ERR_INVALID_ARG, "need 1..64 materials");
    for (int q = 0; q < d->n_materials; q++) {
        const ml_material &m = d->materials[q];
        if (!(m.eps_inf > 0.0) || m.n_extra < 0 || m.n_extra > ML_MAX_POLES - 1)
            return fail(ML_ERR_INVALID_ARG, "material needs eps_inf > 0 and 0 <= n_extra < ML_MAX_POLES");
        for (int p = 0; p <= m.n_extra; p++) {
            const double wp = p ? m.extra[p - 1].wp : m.wp, ga = p ? m.extra[p - 1].gamma : m.gamma,
                         w0 = p ? m.extra[p - 1].omega0 : m.omega0;
            if (!(wp >= 0.0) || !(ga >= 0.0) || !(w0 >= 0.0))
                return fail(ML_ERR_INVALID_ARG, "a pole needs wp >= 0, gamma >= 0, omega0 >= 0");
        }
    }
    if (d->n_sources < 0 || d->n_sources > ML_MAX_SOURCES || (d->n_sources && !d->sources))
        return fail(ML_ERR_INVALID_ARG, "0..4 sources");
    if (d->zchunk < 0 || d->zchunk == 1) return fail(ML_ERR_INVALID_ARG, "zchunk must be 0 (automatic) or >= 2");
    for (int q = 0; q < d->n_sources; q++) {
        const ml_source &s = d->sources[q];
        if (s.axis < 0 || s.axis > 2 || s.comp < 0 || s.comp > 2 || s.comp == s.axis || s.index < 0 ||
            s.index >= dims[s.axis] || !(s.width > 0))
            return fail(ML_ERR_INVALID_ARG, "bad source");
    }
    const long long N = (long long)d->nx * d->ny * d->nz;
    if (d->mat && N >= (1ll << 32)) return fail(ML_ERR_INVALID_ARG, "a material map needs fewer than 2^32 cells");
    if (d->mat)
        for (long long c = 0; c < N; c++)
            if (d->mat[c] >= d->n_materials) return fail(ML_ERR_INVALID_ARG, "material index out of range");
    if (d->design_box[3] > 0) {
        for (int a = 0; a < 3; a++)
            if (d->design_box[a] < 0 || d->design_box[3 + a] < 1 || d->design_box[a] + d->design_box[3 + a] > dims[a])
                return fail(ML_ERR_INVALID_ARG, "design box outside the grid");
        if (!d->design_eps) return fail(ML_ERR_INVALID_ARG, "design box without eps values");
    }

    ml_grid *g = new ml_grid();
    auto bail = [&](ml_status s) {
        cudaDeviceSynchronize();
        dev_free_all(g->allocs);
        delete g;
        return s;
    };
    g->prec = d->precision;
    g->esz = g->prec ? 8 : 4;
    g->nx = d->nx; g->ny = d->ny; g->nz = d->nz;
    g->dt = d->courant;
    for (int a = 0; a < 3; a++) g->per[a] = d->periodic[a] ? 1 : 0;
    for (int f = 0; f < 6; f++) g->pml[f] = d->pml[f];
    g->pml_m = d->pml_m; g->smax = d->pml_sigma_max; g->kmax = d->pml_kappa_max; g->amax = d->pml_alpha_max;
    // tiling and padded layout
    g->ntx = (g->nx + TX - 1) / TX;
    g->nty = (g->ny + TY - 1) / TY;
    int tiles = g->ntx * g->nty;
    // z chunks: the z CPML layers get chunks of their own so that interior chunks
    // take the lean path of the field pass; the interior is split evenly so that
    // the grid has about 8 blocks per SM
    {
        const int target = 8 * 152;
        const int want = std::max(1, std::min((target + tiles - 1) / tiles, (g->nz + 3) / 4));
        const int zl = g->pml[4], zh = g->pml[5];
        // the low layer's chunk also takes the first plane above it: the chunk after it
        // then recomputes, as its z-1 neighbour, a plane outside the layer
        const int zlc = zl > 0 ? std::min(zl + 1, g->nz - zh) : 0;
        std::vector<std::pair<int, int>> seg;
        if (zlc > 0) seg.push_back({0, zlc});
        if (g->nz - zh > zlc) seg.push_back({zlc, g->nz - zh});
        if (zh > 0) seg.push_back({g->nz - zh, g->nz});
        int len = std::min(16, std::max(4, (g->nz + want - 1) / want));
        // a large grid keeps many waves of blocks with 32-plane chunks, which halve the
        // chunks' extra boundary planes and ring fills (measured on the 512 x 512 x 384
        // Bragg ensemble: field pass 1.34 -> 1.25 ms; at 256^3, with four waves, slower)
        if (len == 16 && (long long)tiles * ((g->nz + 31) / 32) >= 12ll * 4 * 152) len = 32;
        // planes per chunk chosen by the caller (shorter chunks shrink the last wave of
        // blocks, longer ones amortise the chunk's extra boundary planes and its ring
        // fill), else the ML_ZCHUNK tuning knob
        if (d->zchunk >= 2) {
            len = d->zchunk;
        } else if (const char *ev = std::getenv("ML_ZCHUNK")) {
            const int v = std::atoi(ev);
            if (v >= 2) len = v;
        }
        g->zcut.assign(1, 0);
        for (auto &sg : seg) {
            const int n = sg.second - sg.first;
            const int pieces = std::max(1, (n + len - 1) / len);
            for (int q = 1; q <= pieces; q++) g->zcut.push_back(sg.first + (int)((long long)n * q / pieces));
        }
        g->nchunk = (int)g->zcut.size() - 1;
        g->cz = 0;
        for (int c = 0; c < g->nchunk; c++) g->cz = std::max(g->cz, g->zcut[c + 1] - g->zcut[c]);
    }
    g->nblocks = tiles * g->nchunk;
    g->px = XO + g->ntx * TX + 32;
    g->py = g->nty * TY + 2;
    g->plane = (long long)g->px * g->py;
    g->vol = (size_t)g->plane * (g->nz + 2);
    ml_status st;
#define GA(ptr, bytes)                                                  \
    do {                                                                \
        st = dalloc(g->allocs, (void **)&(ptr), (bytes));               \
        if (st != ML_OK) return bail(st);                               \
    } while (0)
#define GC(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            fail(ML_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return bail(ML_ERR_CUDA);                                   \
        }                                                               \
    } while (0)
    for (int l = 0; l < 2; l++)
        for (int c = 0; c < 6; c++) GA(g->F[l][c], g->vol * g->esz);
    GA(g->scratch, (size_t)N * 8);
    // CPML tables and memory slabs
    for (int a = 0; a < 3; a++) {
        int n = dims[a];
        std::vector<double> tab(6 * (size_t)n);
        for (int i = 0; i < n; i++) {
            cpml_coeff(g, a, (double)i, tab[i], tab[n + i], tab[2 * n + i]);
            cpml_coeff(g, a, i + 0.5, tab[3 * n + i], tab[4 * n + i], tab[5 * n + i]);
        }
        st = upload_reals(g, g->allocs, &g->cpml[a], tab);
        if (st != ML_OK) return bail(st);
        int th = g->pml[2 * a] + g->pml[2 * a + 1];
        if (th) {
            size_t cnt = (size_t)N / n * th;
            g->psi_n[a] = cnt;
            for (int q = 0; q < 2; q++) {
                GA(g->psiH[0][a][q], cnt * g->esz);
                GA(g->psiH[1][a][q], cnt * g->esz);
                GA(g->psiE[a][q], cnt * g->esz);
            }
        }
    }
    // materials: dt / eps_inf, and per pole slot (material-major, ML_MAX_POLES slots per
    // material) the ADE factors; a material's poles with wp > 0 take slots 0, 1, ...
    std::vector<double> cb(ML_MAX_MATERIALS, g->dt), dk(ML_MAX_MATERIALS * ML_MAX_POLES, 0.0),
        db(ML_MAX_MATERIALS * ML_MAX_POLES, 0.0), dp(ML_MAX_MATERIALS * ML_MAX_POLES, 0.0);
    std::vector<uint8_t> has_pole(ML_MAX_MATERIALS, 0);
    bool any_lorentz = false;
    g->npole = 0;
    for (int q = 0; q < d->n_materials; q++) {
        const ml_material &m = d->materials[q];
        cb[q] = g->dt / m.eps_inf;
        int n = 0;
        for (int p = 0; p <= m.n_extra; p++) {
            const double wp = p ? m.extra[p - 1].wp : m.wp, ga = p ? m.extra[p - 1].gamma : m.gamma,
                         w0 = p ? m.extra[p - 1].omega0 : m.omega0;
            if (!(wp > 0)) continue;
            const double g2 = 0.5 * ga * g->dt;
            const int k = q * ML_MAX_POLES + n++;
            dk[k] = (1.0 - g2) / (1.0 + g2);
            db[k] = wp * wp * g->dt / (1.0 + g2);
            dp[k] = w0 * w0 * g->dt / (1.0 + g2);
            any_lorentz = any_lorentz || w0 > 0;
        }
        has_pole[q] = n > 0;
        g->npole = std::max(g->npole, n);
    }
    st = upload_reals(g, g->allocs, &g->mat_cb, cb);
    if (st != ML_OK) return bail(st);
    st = upload_reals(g, g->allocs, &g->mat_dk, dk);
    if (st != ML_OK) return bail(st);
    st = upload_reals(g, g->allocs, &g->mat_db, db);
    if (st != ML_OK) return bail(st);
    st = upload_reals(g, g->allocs, &g->mat_dp, dp);
    if (st != ML_OK) return bail(st);
    if (d->mat) {
        GA(g->mat, (size_t)N);
        GC(cudaMemcpy(g->mat, d->mat, (size_t)N, cudaMemcpyHostToDevice));
    }
    if (d->design_box[3] > 0) {
        for (int q = 0; q < 6; q++) g->dbox[q] = d->design_box[q];
        size_t cnt = (size_t)g->dbox[3] * g->dbox[4] * g->dbox[5];
        std::vector<double> v(cnt);
        for (size_t q = 0; q < cnt; q++) {
            if (!(d->design_eps[q] > 0.0)) return bail(fail(ML_ERR_INVALID_ARG, "design eps must be > 0"));
            v[q] = g->dt / d->design_eps[q];
        }
        st = upload_reals(g, g->allocs, &g->dcb, v);
        if (st != ML_OK) return bail(st);
    }
    // pole box: bounding box of cells whose material has a dispersive pole
    int lo[3] = {g->nx, g->ny, g->nz}, hi[3] = {-1, -1, -1};
    if (g->npole > 0) {
        for (int k = 0; k < g->nz; k++)
            for (int j = 0; j < g->ny; j++)
                for (int i = 0; i < g->nx; i++) {
                    int q = d->mat ? d->mat[((long long)k * g->ny + j) * g->nx + i] : 0;
                    if (has_pole[q]) {
                        int idx[3] = {i, j, k};
                        for (int a = 0; a < 3; a++) { lo[a] = std::min(lo[a], idx[a]); hi[a] = std::max(hi[a], idx[a]); }
                    }
                }
    }
    if (hi[0] >= 0) {
        for (int a = 0; a < 3; a++) { g->jbox[a] = lo[a]; g->jbox[3 + a] = hi[a] - lo[a] + 1; }
        g->jcnt = (size_t)g->jbox[3] * g->jbox[4] * g->jbox[5];
        GA(g->JD, 3 * (size_t)g->npole * g->jcnt * g->esz);
        if (any_lorentz) GA(g->PD, 3 * (size_t)g->npole * g->jcnt * g->esz);
    }
    for (int l = 0; l < 2; l++)
        for (int c = 0; c < 3; c++) {
            st = make_tmap(g, g->F[l][c], BOXH, &g->tm[l].E[c]);
            if (st != ML_OK) return bail(st);
            st = make_tmap(g, g->F[l][3 + c], BOXHH, &g->tm[l].H[c]);
            if (st != ML_OK) return bail(st);
        }
    GA(g->absorbed_part, (size_t)g->nblocks * sizeof(double));
    GA(g->d_zcut, g->zcut.size() * sizeof(int));
    GC(cudaMemcpy(g->d_zcut, g->zcut.data(), g->zcut.size() * sizeof(int), cudaMemcpyHostToDevice));
    GA(g->d_scalar, 64 * sizeof(double));
    GA(g->d_fpart, (size_t)ML_MAX_FREQS * FLUX_NB * sizeof(double));
    GA(g->d_status, sizeof(int));
    for (int q = 0; q < d->n_sources; q++) {
        const ml_source &s = d->sources[q];
        g->src.push_back(SrcDev{s.axis, s.index, s.comp, s.amp, s.omega, s.width, s.t0});
    }
    {
        // per-tile work of the field pass's own cells: bit 0 = the design box or the pole
        // box, bit 1 = a non-background material, bit 2 = a source plane
        std::vector<int> zt(g->nz);
        for (int c = 0; c < g->nchunk; c++)
            for (int k = g->zcut[c]; k < g->zcut[c + 1]; k++) zt[k] = c;
        std::vector<uint8_t> fl((size_t)g->nblocks, 0);
        auto tile_of = [&](int i, int j, int k) { return ((long long)zt[k] * g->nty + j / TY) * g->ntx + i / TX; };
        if (d->mat)
            for (int k = 0; k < g->nz; k++)
                for (int j = 0; j < g->ny; j++)
                    for (int i = 0; i < g->nx; i++)
                        if (d->mat[((long long)k * g->ny + j) * g->nx + i] != 0) fl[tile_of(i, j, k)] |= 2;
        for (int bz = 0; bz < g->nchunk; bz++)
            for (int by = 0; by < g->nty; by++)
                for (int bx = 0; bx < g->ntx; bx++) {
                    const int lo[3] = {bx * TX, by * TY, g->zcut[bz]};
                    const int hi[3] = {std::min(g->nx, bx * TX + TX), std::min(g->ny, by * TY + TY), g->zcut[bz + 1]};
                    auto meets = [&](const int *box) {
                        if (box[3] <= 0) return false;
                        for (int a = 0; a < 3; a++)
                            if (box[a] >= hi[a] || box[a] + box[3 + a] <= lo[a]) return false;
                        return true;
                    };
                    uint8_t f = (meets(g->dbox) || meets(g->jbox)) ? 1 : 0;
                    for (auto &q : g->src)
                        if (q.index >= lo[q.axis] && q.index < hi[q.axis]) f |= 4;
                    fl[((long long)bz * g->nty + by) * g->ntx + bx] |= f;
                }
        GA(g->d_tflags, fl.size());
        GC(cudaMemcpy(g->d_tflags, fl.data(), fl.size(), cudaMemcpyHostToDevice));
    }
    {
        // Which field-pass bodies the grid's tiles take (block_mode, evaluated once on the
        // device): a grid whose tiles need only the interior and CPML bodies, or only the
        // interior and table bodies, gets a field-pass kernel compiled with those alone.
        // The five bodies together are more code than the SM keeps close at hand, and the
        // smaller kernels measured faster (256^3 vacuum slab 227 -> 216 us per pass).
        GA(g->d_tmode, (size_t)g->nblocks);
        cudaError_t e;
        if (g->prec) {
            YeeArgs<double> y;
            fill_yee_args<double>(g, 0, y);
            e = launch_tile_modes<double>(y, g->nblocks, g->d_tmode, 0);
        } else {
            YeeArgs<float> y;
            fill_yee_args<float>(g, 0, y);
            e = launch_tile_modes<float>(y, g->nblocks, g->d_tmode, 0);
        }
        GC(e);
        std::vector<uint8_t> md((size_t)g->nblocks);
        GC(cudaMemcpy(md.data(), g->d_tmode, md.size(), cudaMemcpyDeviceToHost));
        bool used[5] = {};
        for (uint8_t m : md) used[m < 5 ? m : 2] = true;
        if (used[2]) g->bodies = YEE_BODIES_ALL;
        else if (used[3] || used[4]) g->bodies = YEE_BODIES_TABLES;
        else g->bodies = YEE_BODIES_VACUUM;
        if (const char *ev = std::getenv("ML_YEE_BODIES"))
            if (std::atoi(ev) == YEE_BODIES_ALL) g->bodies = YEE_BODIES_ALL;
    }
    GC(cudaDeviceSynchronize());
    *out = g;
    return ML_OK;
#undef GA
#undef GC
}

// ------------------------------------------------------------------ molecules

namespace {

ml_status rebuild_molecules(ml_grid *g) {
    cudaDeviceSynchronize();
    dev_free_all(g->mol_allocs);
    auto &L = g->mol_allocs;
    const int M = g->nmol;
    ml_status st;
    // every molecule two-level: the pool offsets are then 4 m (pools are appended in order)
    g->two_level = std::all_of(g->nlev.begin(), g->nlev.end(), [](int n) { return n == 2; });
#define CKS(x)                     \
    do {                           \
        st = (x);                  \
        if (st != ML_OK) return st; \
    } while (0)
    CKS(upload_raw(L, &g->d_nlev, g->nlev));
    CKS(upload_raw(L, &g->d_kind, g->kind));
    CKS(upload_raw(L, &g->d_nsub, g->nsub));
    CKS(upload_raw(L, &g->d_cmask, g->cmask));
    CKS(upload_raw(L, &g->d_win, g->win));
    CKS(upload_raw(L, &g->d_wf, g->wf));
    CKS(upload_raw(L, &g->d_wraw, g->wraw));
    CKS(upload_raw(L, &g->d_off, g->off));
    CKS(upload_raw(L, &g->d_pos, g->pos));
    CKS(upload_raw(L, &g->d_sigma, g->sigma));
    CKS(upload_reals(g, L, &g->d_gamma, g->gamma));
    CKS(upload_reals(g, L, &g->d_decay, g->decay));
    CKS(upload_reals(g, L, &g->d_deph, g->deph));
    CKS(upload_reals(g, L, &g->d_H0, g->H0));
    CKS(upload_reals(g, L, &g->d_mu, g->mu));
    CKS(upload_reals(g, L, &g->d_rho, g->rho0));
    AL(L, g->d_w, (size_t)M * NW * g->esz);
    AL(L, g->d_Et, (size_t)M * 3 * g->esz);
    AL(L, g->d_mudot, (size_t)M * 3 * g->esz);
    AL(L, g->d_c, (size_t)M * 3 * g->esz);
    AL(L, g->d_energy, (size_t)M * sizeof(double));
    AL(L, g->d_export, std::max<size_t>((size_t)std::max<long long>(2 * g->pool, (long long)M * MAXLEV), 1) * sizeof(double));
    const int dims[3] = {g->nx, g->ny, g->nz};
    cudaError_t e = g->prec ? launch_weights<double>(M, g->d_pos, g->d_sigma, g->d_win, g->d_wf, g->d_wraw, dims,
                                                     g->per, (double *)g->d_w, 0)
                            : launch_weights<float>(M, g->d_pos, g->d_sigma, g->d_win, g->d_wf, g->d_wraw, dims,
                                                    g->per, (float *)g->d_w, 0);
    if (e != cudaSuccess) return fail(ML_ERR_CUDA, std::string("weights kernel: ") + cudaGetErrorString(e));
    // box of the molecular current: bounding box of the (folded) kernel windows;
    // an axis on which some window wraps around a periodic boundary is taken whole
    g->gcmask = 0;
    for (int m = 0; m < M; m++) g->gcmask |= g->cmask[m];
    for (int a = 0; a < 3; a++) {
        const int n = dims[a];
        int lo = n, hi = 0;
        bool whole = false;
        for (int m = 0; m < M; m++) {
            const int Wf = (g->wf[m] >> (8 * a)) & 0xff;
            const int st0 = g->win[3 * m + a];
            if (st0 + Wf > n) whole = true;
            lo = std::min(lo, st0);
            hi = std::max(hi, st0 + Wf);
        }
        if (whole || M == 0) { lo = 0; hi = n; }
        g->jb0[a] = lo;
        g->jbn[a] = std::max(0, hi - lo);
    }
    g->jnbx = (g->jbn[0] + JX - 1) / JX;
    g->jnby = (g->jbn[1] + JY - 1) / JY;
    const int jnbz = (g->jbn[2] + JZ - 1) / JZ;
    g->jnb = g->jnbx * g->jnby * jnbz;
    // entries (m, window start relative to the block origin) of every block a window
    // touches, in molecule order
    std::vector<std::vector<int4>> lists(g->jnb);
    for (int m = 0; m < M; m++) {
        std::vector<std::pair<int, int>> ax[3];  // (block coordinate, local start)
        for (int a = 0; a < 3; a++) {
            const int n = dims[a];
            const int Wf = (g->wf[m] >> (8 * a)) & 0xff;
            const int st0 = g->win[3 * m + a];
            const int T_ = a == 0 ? JX : (a == 1 ? JY : JZ);
            const int nbk = a == 0 ? g->jnbx : (a == 1 ? g->jnby : jnbz);
            int copies[2] = {st0, st0 - n};
            const int ncopy = g->per[a] ? 2 : 1;
            for (int q = 0; q < ncopy; q++) {
                const int s0 = copies[q] - g->jb0[a];
                const int c0 = std::max(s0, 0), c1 = std::min(s0 + Wf, g->jbn[a]);
                if (c0 >= c1) continue;
                for (int b = c0 / T_; b <= (c1 - 1) / T_ && b < nbk; b++) ax[a].push_back({b, s0 - b * T_});
            }
        }
        for (auto &z : ax[2])
            for (auto &y : ax[1])
                for (auto &x : ax[0])
                    lists[(z.first * g->jnby + y.first) * g->jnbx + x.first].push_back(make_int4(m, x.second, y.second, z.second));
    }
    std::vector<int> joff(g->jnb + 1, 0);
    std::vector<int4> jent;
    for (int b = 0; b < g->jnb; b++) {
        joff[b] = (int)jent.size();
        jent.insert(jent.end(), lists[b].begin(), lists[b].end());
    }
    joff[g->jnb] = (int)jent.size();
    CKS(upload_raw(L, &g->d_joff, joff));
    if (!jent.empty()) CKS(upload_raw(L, &g->d_jent, jent));
    {
        std::vector<unsigned char> jmask(jent.size());
        for (size_t e = 0; e < jent.size(); e++) {
            const int lo = jent[e].y, hi = lo + (g->wf[jent[e].x] & 0xff);
            unsigned mk = 0;
            for (int q = 0; q < JX / 4; q++)
                if (lo < 4 * q + 4 && hi > 4 * q) mk |= 1u << q;
            jmask[e] = (unsigned char)mk;
        }
        if (!jmask.empty()) CKS(upload_raw(L, &g->d_jmask, jmask));
    }
    // molecule -> entries (ascending entry index)
    std::vector<int> moff(M + 1, 0), mlist(jent.size());
    for (const int4 &e : jent) moff[e.x + 1]++;
    for (int m = 0; m < M; m++) moff[m + 1] += moff[m];
    {
        std::vector<int> fill(moff.begin(), moff.end() - 1);
        for (int e = 0; e < (int)jent.size(); e++) mlist[fill[jent[e].x]++] = e;
    }
    CKS(upload_raw(L, &g->d_moff, moff));

    if (!mlist.empty()) CKS(upload_raw(L, &g->d_mlist, mlist));
    AL(L, g->d_part, std::max<size_t>(jent.size(), 1) * 3 * g->esz);
    // field-pass blocks whose tile (with halo) meets the current box
    {
        std::vector<int> A, B;
        for (int t = 0; t < g->nblocks; t++) {
            const int bx = t % g->ntx, by = (t / g->ntx) % g->nty, bz = t / (g->ntx * g->nty);
            const int x0 = bx * TX, y0 = by * TY, k0 = g->zcut[bz], k1 = g->zcut[bz + 1];
            const bool hit = g->gcmask && x0 - 1 < g->jb0[0] + g->jbn[0] && x0 + TX > g->jb0[0] &&
                             y0 - 1 < g->jb0[1] + g->jbn[1] && y0 + TY > g->jb0[1] && k0 - 1 < g->jb0[2] + g->jbn[2] &&
                             k1 > g->jb0[2];
            (hit ? B : A).push_back(t);
        }
        g->nblA = (int)A.size();
        g->nblB = (int)B.size();
        if (!A.empty()) CKS(upload_raw(L, &g->d_blA, A));
        if (!B.empty()) CKS(upload_raw(L, &g->d_blB, B));
    }
    if (const char *ev = std::getenv("ML_OVERLAP")) g->overlap = std::atoi(ev) != 0;
    if (const char *ev = std::getenv("ML_PDL")) g->pdl = std::atoi(ev) != 0;
    if (!g->side) {
        // highest priority: the chain's short kernels take SMs as field-pass blocks retire
        int lowest = 0, highest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&lowest, &highest));
        CK(cudaStreamCreateWithPriority(&g->side, cudaStreamNonBlocking, highest));
        CK(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&g->ev_box, cudaEventDisableTiming));
    }
    const size_t jvol = (size_t)g->jbn[0] * g->jbn[1] * g->jbn[2];
    for (int c = 0; c < 3; c++) {
        g->d_J[c] = nullptr;
        if ((g->gcmask >> c) & 1) AL(L, g->d_J[c], jvol * g->esz);
    }
    // packed molecule kernel (grids with multilevel molecules): molecules sorted by
    // (kind, level count, substeps) and, within a class, by the 16-cell brick of their
    // window start, then by window position (consecutive items run on the same SM, and
    // their windows overlap: 0.2360 -> 0.2341 ms on the 512 x 512 x 384 ensemble against
    // the plain z, y, x order), cut into work items of pack_per_warp(n) molecules.  (Bands
    // of z first, to keep one band of the field in L2 for every class, measured slower:
    // 0.236 -> 0.249 ms, warps of one block then run different level counts.)
    g->nitems = 0;
    if (!g->two_level && M > 0) {
        std::vector<int> ord(M);
        for (int m = 0; m < M; m++) ord[m] = m;
        auto key = [&](int m) {
            return std::make_tuple(g->kind[m] == 0 ? 0 : 1, g->nlev[m], g->nsub[m], g->win[3 * m + 2] / 16,
                                   g->win[3 * m + 1] / 16, g->win[3 * m] / 16, g->win[3 * m + 2],
                                   g->win[3 * m + 1], g->win[3 * m], m);
        };
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return key(x) < key(y); });
        std::vector<int4> items;
        for (int i = 0; i < M;) {
            const int m0 = ord[i];
            const int n = g->nlev[m0], cls = g->kind[m0] == 0 ? 0 : 1, ns = g->nsub[m0];
            const int per = pack_per_warp(n);
            int c = 0;
            while (i + c < M && c < per) {
                const int mc = ord[i + c];
                if (g->nlev[mc] != n || (g->kind[mc] == 0 ? 0 : 1) != cls || g->nsub[mc] != ns) break;
                c++;
            }
            items.push_back(make_int4(i, c, n, cls | (ns << 4)));
            i += c;
        }
        g->nitems = (int)items.size();
        CKS(upload_raw(L, &g->d_order, ord));
        CKS(upload_raw(L, &g->d_items, items));
    }
    CK(cudaDeviceSynchronize());
    return ML_OK;
#undef CKS
}

}  // namespace

ml_status ml_add_molecules(ml_grid *g, const ml_molecule_desc *md, void *stream, int *first_id) {
    (void)stream;
    if (!g || !md) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (md->count < 0) return fail(ML_ERR_INVALID_ARG, "negative count");
    if (md->count == 0) {
        if (first_id) *first_id = g->nmol;
        return ML_OK;
    }
    if (!md->nlev || !md->off || !md->pos || !md->sigma || !md->gamma || !md->decay || !md->dephase ||
        !md->kind || !md->nsub || !md->H0 || !md->mu || !md->rho)
        return fail(ML_ERR_INVALID_ARG, "null molecule array");
    const int dims[3] = {g->nx, g->ny, g->nz};
    // keep the evolving state of molecules added earlier
    if (g->nmol > 0 && g->step > 0) {
        std::vector<double> buf(2 * g->pool);
        ml_status s = ml_get_molecules(g, ML_MOL_RHO, buf.data(), 0, nullptr);
        if (s != ML_OK) return s;
        g->rho0 = buf;
    }
    const long long base = g->pool;
    for (int m = 0; m < md->count; m++) {
        int n = md->nlev[m];
        if (n < 2 || n > ML_MAX_LEVELS) return fail(ML_ERR_INVALID_ARG, "nlev must be 2..8");
        if (md->off[m] < 0 || md->off[m] + (long long)n * n > md->pool) return fail(ML_ERR_INVALID_ARG, "pool offset out of range");
        if (md->kind[m] != 0 && md->kind[m] != 1) return fail(ML_ERR_INVALID_ARG, "kind must be 0 or 1");
        if (md->kind[m] == 0 && (n != 2 || md->decay[m] != 0.0 || md->dephase[m] != 0.0))
            return fail(ML_ERR_INVALID_ARG, "kind 0 needs two levels and no Lindblad terms");
        if (md->nsub[m] < 1) return fail(ML_ERR_INVALID_ARG, "nsub must be >= 1");
        if (!(md->sigma[m] > 0.0) || std::ceil(3.0 * md->sigma[m]) > 7.0)
            return fail(ML_ERR_INVALID_ARG, "sigma must be in (0, 7/3]");
        if (md->decay[m] < 0.0 || md->dephase[m] < 0.0) return fail(ML_ERR_INVALID_ARG, "negative rate");
        int R = (int)std::ceil(3.0 * md->sigma[m]);
        int W = 2 * R + 2;
        int wfp = 0;
        int wstart[3];
        for (int a = 0; a < 3; a++) {
            double p = md->pos[3 * m + a];
            if (!std::isfinite(p)) return fail(ML_ERR_INVALID_ARG, "non-finite position");
            long long s = (long long)std::floor(p) - R;
            int n_ = dims[a];
            int Wf;
            if (g->per[a]) {
                long long sc = ((s % n_) + n_) % n_;
                wstart[a] = (int)sc;
                Wf = std::min(W, n_);
            } else {
                if (s < 0 || s + W > n_)
                    return fail(ML_ERR_INVALID_ARG, "molecule " + std::to_string(m) + ": kernel window crosses a wall");
                wstart[a] = (int)s;
                Wf = W;
            }
            wfp |= Wf << (8 * a);
        }
        int cm = 0;
        for (int c = 0; c < 3; c++)
            for (int e = 0; e < n * n; e++) {
                const double *z = md->mu + 2 * (c * md->pool + md->off[m] + e);
                if (z[0] != 0.0 || z[1] != 0.0) cm |= 1 << c;
            }
        g->nlev.push_back(n);
        g->off.push_back(g->pool);
        g->kind.push_back(md->kind[m]);
        g->nsub.push_back(md->nsub[m]);
        g->cmask.push_back(cm);
        for (int a = 0; a < 3; a++) {
            g->win.push_back(wstart[a]);
            g->wraw.push_back(W);
            g->pos.push_back(md->pos[3 * m + a]);
        }
        g->wf.push_back(wfp);
        g->sigma.push_back(md->sigma[m]);
        g->gamma.push_back(md->gamma[m]);
        g->decay.push_back(md->decay[m]);
        g->deph.push_back(md->dephase[m]);
        g->pool += (long long)n * n;
    }
    // pools (append)
    std::vector<double> mu_new(2 * 3 * (size_t)g->pool, 0.0);
    for (int c = 0; c < 3; c++) {
        long long oldp = base;
        for (long long e = 0; e < oldp; e++) {
            mu_new[2 * (c * g->pool + e)] = g->mu.empty() ? 0.0 : g->mu[2 * (c * oldp + e)];
            mu_new[2 * (c * g->pool + e) + 1] = g->mu.empty() ? 0.0 : g->mu[2 * (c * oldp + e) + 1];
        }
    }
    long long w = base;
    for (int m = 0; m < md->count; m++) {
        int nn = md->nlev[m] * md->nlev[m];
        for (int e = 0; e < nn; e++) {
            long long src = md->off[m] + e;
            g->H0.push_back(md->H0[2 * src]);
            g->H0.push_back(md->H0[2 * src + 1]);
            g->rho0.push_back(md->rho[2 * src]);
            g->rho0.push_back(md->rho[2 * src + 1]);
            for (int c = 0; c < 3; c++) {
                mu_new[2 * (c * g->pool + w + e)] = md->mu[2 * (c * md->pool + src)];
                mu_new[2 * (c * g->pool + w + e) + 1] = md->mu[2 * (c * md->pool + src) + 1];
            }
        }
        w += nn;
    }
    g->mu.swap(mu_new);
    std::vector<double> energy_keep;
    if (g->nmol > 0 && g->d_energy) {
        energy_keep.resize(g->nmol);
        CK(cudaMemcpy(energy_keep.data(), g->d_energy, g->nmol * sizeof(double), cudaMemcpyDeviceToHost));
    }
    int first = g->nmol;
    g->nmol += md->count;
    ml_status s = rebuild_molecules(g);
    if (s != ML_OK) return s;
    if (!energy_keep.empty())
        CK(cudaMemcpy(g->d_energy, energy_keep.data(), energy_keep.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (first_id) *first_id = first;
    return ML_OK;
}

ml_status ml_add_flux_plane(ml_grid *g, int axis, int index, int nfreq, const double *omega, int *id) {
    if (!g || !omega) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (axis < 0 || axis > 2) return fail(ML_ERR_INVALID_ARG, "axis must be 0..2");
    if (index < 0 || index >= dim(g, axis)) return fail(ML_ERR_INVALID_ARG, "plane index out of range");
    if (nfreq < 1 || nfreq > ML_MAX_FREQS) return fail(ML_ERR_INVALID_ARG, "nfreq must be 1..64");
    if (g->nsamp != 0) return fail(ML_ERR_STATE, "planes must be added between folds (before stepping)");
    if ((int)g->planes.size() >= MAXPLANES) return fail(ML_ERR_INVALID_ARG, "at most 8 flux planes");
    Plane p;
    p.axis = axis;
    p.index = index;
    p.nfreq = nfreq;
    p.nb = dim(g, (axis + 1) % 3);
    p.nc = dim(g, (axis + 2) % 3);
    p.omega.assign(omega, omega + nfreq);
    ml_status st = upload_raw(g->allocs, &p.d_omega, p.omega);
    if (st != ML_OK) return st;
    size_t ncell = (size_t)p.nb * p.nc;
    AL(g->allocs, p.d_buf, (size_t)DFT_KMAX * 4 * ncell * g->esz);
    AL(g->allocs, p.d_acc, 4 * (size_t)nfreq * ncell * sizeof(double2));
    AL(g->allocs, p.d_ph, 2 * (size_t)DFT_KMAX * nfreq * g->esz);
    {
        cudaError_t e = g->prec ? launch_dft_phases<double>(p.d_omega, nfreq, g->dt, (double *)p.d_ph, 0)
                                : launch_dft_phases<float>(p.d_omega, nfreq, g->dt, (float *)p.d_ph, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(ML_ERR_CUDA, std::string("phase table: ") + cudaGetErrorString(e));
    }
    g->planes.push_back(p);
    if (id) *id = (int)g->planes.size() - 1;
    return ML_OK;
}

// ------------------------------------------------------------------ stepping

namespace ml {

template <typename T>
ml_status fold_planes(ml_grid *g, cudaStream_t s) {
    if (g->nsamp == 0) return ML_OK;
    for (auto &p : g->planes) {
        LaunchScope ls(g, s, 3);
        CK(launch_dft_fold<T>((const T *)p.d_buf, g->nsamp, p.nb * p.nc, p.nfreq, p.d_omega, (const T *)p.d_ph,
                              g->samp_step0, g->dt, p.d_acc, s));
    }
    g->nsamp = 0;
    return ML_OK;
}

template <typename T>
void fill_mol_args(ml_grid *g, int cur, MolArgs<T> &m) {
    m = MolArgs<T>{};
    m.nmol = g->nmol;
    m.dt = (T)g->dt;
    m.nx = g->nx; m.ny = g->ny; m.nz = g->nz; m.px = g->px; m.plane = g->plane;
    for (int a = 0; a < 3; a++) { m.per[a] = g->per[a]; m.E[a] = (const T *)g->F[cur][a]; }
    m.nlev = g->d_nlev; m.off = g->d_off; m.kind = g->d_kind; m.nsub = g->d_nsub; m.cmask = g->d_cmask;
    m.gamma = (const T *)g->d_gamma; m.decay = (const T *)g->d_decay; m.dephase = (const T *)g->d_deph;
    m.H0 = (const cx<T> *)g->d_H0; m.mu = (const cx<T> *)g->d_mu; m.pool = g->pool;
    m.rho = (cx<T> *)g->d_rho;
    m.Et = (T *)g->d_Et; m.mudot = (T *)g->d_mudot; m.c = (T *)g->d_c;
    m.energy = g->d_energy; m.status = g->d_status;
    m.win = g->d_win; m.wf = g->d_wf; m.w = (const T *)g->d_w;
    m.two_level = g->two_level ? 1 : 0;
    m.order = g->d_order;
    m.items = g->d_items;
    m.nitems = g->nitems;
    m.pop_sink = g->pop_off ? nullptr : g->pop_sink;
    m.pop_slot = g->pop_sink ? (g->step % g->pop_ring) * (long long)g->nmol * MAXLEV : 0;
}

template <typename T>
void fill_gath_args(ml_grid *g, int cur, GathArgs<T> &ga) {
    ga = GathArgs<T>{};
    ga.nblocks = g->jnb; ga.nbx = g->jnbx; ga.nby = g->jnby;
    for (int q = 0; q < 3; q++) { ga.bn[q] = g->jbn[q]; ga.b0[q] = g->jb0[q]; ga.E[q] = (const T *)g->F[cur][q]; }
    ga.px = g->px; ga.plane = g->plane;
    ga.off = g->d_joff; ga.ent = g->d_jent; ga.wf = g->d_wf; ga.w = (const T *)g->d_w; ga.cmask = g->d_cmask;
    ga.gcmask = g->gcmask; ga.part = (T *)g->d_part;
}

template <typename T>
void fill_cur_args(ml_grid *g, CurArgs<T> &ca) {
    ca = CurArgs<T>{};
    ca.nblocks = g->jnb; ca.nbx = g->jnbx; ca.nby = g->jnby;
    for (int a = 0; a < 3; a++) ca.bn[a] = g->jbn[a];
    ca.off = g->d_joff; ca.ent = g->d_jent; ca.emask = g->d_jmask; ca.wf = g->d_wf; ca.w = (const T *)g->d_w;
    ca.c = (const T *)g->d_c; ca.cmask = g->gcmask;
    for (int c = 0; c < 3; c++) ca.J[c] = (T *)g->d_J[c];
}

// Arguments of the field pass reading level `cur`, with the DFT ring at slot 0.
template <typename T>
void fill_yee_args(ml_grid *g, int cur, YeeArgs<T> &y) {
    const int nxt = cur ^ 1;
    y = YeeArgs<T>{};
    y.nx = g->nx; y.ny = g->ny; y.nz = g->nz; y.px = g->px; y.py = g->py; y.plane = g->plane;
    for (int a = 0; a < 3; a++) y.per[a] = g->per[a];
    for (int f = 0; f < 6; f++) y.pml[f] = g->pml[f];
    y.ntx = g->ntx; y.nty = g->nty; y.nchunk = g->nchunk; y.cz = g->cz; y.zcut = g->d_zcut;
    y.tflags = g->d_tflags;
    y.bodies = g->bodies;
    y.dt = (T)g->dt;
    for (int c = 0; c < 3; c++) {
        y.Eo[c] = (const T *)g->F[cur][c];
        y.Ho[c] = (const T *)g->F[cur][3 + c];
        y.En[c] = (T *)g->F[nxt][c];
        y.Hn[c] = (T *)g->F[nxt][3 + c];
    }
    for (int a = 0; a < 3; a++) {
        y.cpml[a] = (const T *)g->cpml[a];
        for (int q = 0; q < 2; q++) {
            y.psiHo[a][q] = (const T *)g->psiH[cur][a][q];
            y.psiHn[a][q] = (T *)g->psiH[nxt][a][q];
            y.psiE[a][q] = (T *)g->psiE[a][q];
        }
    }
    y.mat = g->mat;
    y.mat_cb = (const T *)g->mat_cb; y.mat_dk = (const T *)g->mat_dk; y.mat_db = (const T *)g->mat_db;
    for (int q = 0; q < 6; q++) { y.dbox[q] = g->dbox[q]; y.jbox[q] = g->jbox[q]; }
    y.dcb = (const T *)g->dcb;
    y.mat_dp = (const T *)g->mat_dp;
    y.npole = g->npole;
    y.jcnt = (long long)g->jcnt;
    y.JD = (T *)g->JD;
    y.PD = (T *)g->PD;
    y.absorbed_part = g->absorbed_part;
    y.status = g->d_status;
    y.wait_limit = g->wait_limit;
    if (g->nmol > 0)
        for (int a = 0; a < 3; a++) {
            y.jb0[a] = g->jb0[a];
            y.jbn[a] = g->jbn[a];
            y.Jb[a] = (const T *)g->d_J[a];
        }
    y.nsrc = (int)g->src.size();
    for (int q = 0; q < y.nsrc; q++) y.src[q] = g->src[q];
    y.step = g->step;
    y.nplanes = (int)g->planes.size();
    for (int p = 0; p < y.nplanes; p++) {
        const Plane &pl = g->planes[p];
        y.planes[p].axis = pl.axis;
        y.planes[p].index = pl.index;
        y.planes[p].nb = pl.nb;
        y.planes[p].nc = pl.nc;
        y.planes[p].buf = (T *)pl.d_buf;
    }
}

// Arguments of the periodic-image refresh of the six field arrays of level `lev`.
template <typename T>
ImgArgs<T> image_args(const ml_grid *g, int lev) {
    ImgArgs<T> a{};
    for (int c = 0; c < 6; c++) a.f[c] = (T *)g->F[lev][c];
    a.nx = g->nx; a.ny = g->ny; a.nz = g->nz; a.px = g->px; a.plane = g->plane;
    for (int q = 0; q < 3; q++) a.per[q] = g->per[q];
    return a;
}

template <typename T>
ml_status step_impl(ml_grid *g, long long nsteps, cudaStream_t s) {
    for (long long it = 0; it < nsteps; it++) {
        const int cur = g->cur, nxt = cur ^ 1;
        // the molecule chain (gather -> molecules -> current) runs on the side stream,
        // forked from everything enqueued on s so far
        const bool chain = g->nmol > 0 && g->overlap;
        cudaStream_t cs = chain ? g->side : s;
        if (chain) {
            CK(cudaEventRecord(g->ev_box, s));
            CK(cudaStreamWaitEvent(g->side, g->ev_box, 0));
        }
        if (g->nmol > 0) {
            {
                // each molecule's warp gathers its regularised field from E^n itself
                MolArgs<T> m;
                fill_mol_args<T>(g, cur, m);
                // programmatic dependent of the previous field pass only when that pass has
                // tiles that read J: such a tile releases this kernel only after its wait
                // for the previous current kernel, hence after the previous molecule
                // kernel, so the molecule state may be staged before this kernel's wait
                const bool pdl_mol = !chain && g->pdl && g->gcmask != 0;
                if (g->nitems > 0) {
                    LaunchScope ls(g, cs, 0);
                    CK(launch_molecules_packed<T>(m, cs, pdl_mol));
                } else {
                    LaunchScope ls(g, cs, 0);
                    CK(launch_molecules<T>(m, cs, pdl_mol));
                }
            }
            {
                CurArgs<T> ca;
                fill_cur_args<T>(g, ca);
                LaunchScope ls(g, cs, 4);
                CK(launch_current<T>(ca, cs, !chain && g->pdl));
            }
            if (chain) CK(cudaEventRecord(g->ev_join, cs));
        }
        YeeArgs<T> y;
        fill_yee_args<T>(g, cur, y);
        if (!g->planes.empty() && g->nsamp == 0) g->samp_step0 = g->step;
        for (int p = 0; p < y.nplanes; p++)
            y.planes[p].buf += (size_t)g->nsamp * 4 * y.planes[p].nb * y.planes[p].nc;
        if (chain) {
            // blocks clear of the current box overlap the chain; the others wait for J
            if (g->nblA > 0) {
                y.blist = g->d_blA;
                LaunchScope ls(g, s, 1);
                CK(launch_yee<T>(y, g->tm[cur], g->nblA, s));
            }
            CK(cudaStreamWaitEvent(s, g->ev_join, 0));
            if (g->nblB > 0) {
                y.blist = g->d_blB;
                LaunchScope ls(g, s, 1);
                CK(launch_yee<T>(y, g->tm[cur], g->nblB, s));
            }
        } else {
            LaunchScope ls(g, s, 1);
            CK(launch_yee<T>(y, g->tm[cur], g->nblocks, s, g->nmol > 0 && g->pdl));
        }
        if (g->per[0] | g->per[1] | g->per[2]) {
            // periodic images of the level just written, before anything reads its ghosts
            LaunchScope ls(g, s, 1);
            CK(launch_images<T>(image_args<T>(g, nxt), s));
        }
        if (!g->planes.empty()) {
            g->nsamp++;
            if (g->nsamp == DFT_KMAX) {
                ml_status st = fold_planes<T>(g, s);
                if (st != ML_OK) return st;
            }
        }
        g->cur = nxt;
        g->step++;
    }
    return ML_OK;
}

template ml_status fold_planes<float>(ml_grid *, cudaStream_t);
template ml_status fold_planes<double>(ml_grid *, cudaStream_t);
template ml_status step_impl<float>(ml_grid *, long long, cudaStream_t);
template ml_status step_impl<double>(ml_grid *, long long, cudaStream_t);
#define ML_FILL(T)                                                    \
    template void fill_mol_args<T>(ml_grid *, int, MolArgs<T> &);     \
    template void fill_gath_args<T>(ml_grid *, int, GathArgs<T> &);   \
    template void fill_cur_args<T>(ml_grid *, CurArgs<T> &);          \
    template void fill_yee_args<T>(ml_grid *, int, YeeArgs<T> &);                                               \
    template ImgArgs<T> image_args<T>(const ml_grid *, int);
ML_FILL(float)
ML_FILL(double)

}  // namespace ml

ml_status ml_step(ml_grid *g, int64_t nsteps, void *stream) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    if (nsteps < 0) return fail(ML_ERR_INVALID_ARG, "negative step count");
    cudaStream_t s = (cudaStream_t)stream;
    return g->prec ? step_impl<double>(g, nsteps, s) : step_impl<float>(g, nsteps, s);
}

// ------------------------------------------------------------------ state access

namespace {
const unsigned kMaskBits[6] = {ML_EX, ML_EY, ML_EZ, ML_HX, ML_HY, ML_HZ};
}

ml_status ml_get_fields(ml_grid *g, unsigned mask, void *dst, int dst_on_device, void *stream) {
    if (!g || !dst) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (mask == 0 || (mask & ~63u)) return fail(ML_ERR_INVALID_ARG, "bad component mask");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    char *out = (char *)dst;
    for (int c = 0; c < 6; c++) {
        if (!(mask & kMaskBits[c])) continue;
        void *tgt = dst_on_device ? (void *)out : g->scratch;
        cudaError_t e = g->prec ? launch_pack_fields<double>((const double *)g->F[g->cur][c], (double *)tgt, g->nx, g->ny,
                                                             g->nz, g->px, g->plane, 0, s)
                                : launch_pack_fields<float>((const float *)g->F[g->cur][c], (float *)tgt, g->nx, g->ny,
                                                            g->nz, g->px, g->plane, 0, s);
        CK(e);
        if (!dst_on_device) CK(cudaMemcpyAsync(out, g->scratch, N * g->esz, cudaMemcpyDeviceToHost, s));
        out += N * g->esz;
    }
    if (!dst_on_device) CK(cudaStreamSynchronize(s));
    return ML_OK;
}

ml_status ml_set_fields(ml_grid *g, unsigned mask, const void *src, int src_on_device, void *stream) {
    if (!g || !src) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (mask == 0 || (mask & ~63u)) return fail(ML_ERR_INVALID_ARG, "bad component mask");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)g->nx * g->ny * g->nz;
    const char *in = (const char *)src;
    for (int c = 0; c < 6; c++) {
        if (!(mask & kMaskBits[c])) continue;
        const void *from = in;
        if (!src_on_device) {
            CK(cudaMemcpyAsync(g->scratch, in, N * g->esz, cudaMemcpyHostToDevice, s));
            from = g->scratch;
        }
        cudaError_t e = g->prec ? launch_pack_fields<double>((const double *)from, (double *)g->F[g->cur][c], g->nx,
                                                             g->ny, g->nz, g->px, g->plane, 1, s)
                                : launch_pack_fields<float>((const float *)from, (float *)g->F[g->cur][c], g->nx,
                                                            g->ny, g->nz, g->px, g->plane, 1, s);
        CK(e);
        e = g->prec ? launch_refresh_ghosts<double>((double *)g->F[g->cur][c], g->nx, g->ny, g->nz, g->px, g->plane,
                                                    g->per, s)
                    : launch_refresh_ghosts<float>((float *)g->F[g->cur][c], g->nx, g->ny, g->nz, g->px, g->plane,
                                                   g->per, s);
        CK(e);
        in += N * g->esz;
        if (!src_on_device) CK(cudaStreamSynchronize(s));  // scratch is reused
    }
    return ML_OK;
}

ml_status ml_set_population_sink(ml_grid *g, double *host, int64_t ring_steps) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    if (!host) {
        g->pop_sink = nullptr;
        g->pop_ring = 0;
        return ML_OK;
    }
    if (ring_steps < 1) return fail(ML_ERR_INVALID_ARG, "ring_steps must be >= 1");
    void *dev = nullptr;
    cudaError_t e = cudaHostGetDevicePointer(&dev, host, 0);
    if (e != cudaSuccess || !dev) {
        cudaGetLastError();
        return fail(ML_ERR_INVALID_ARG, "the population sink must be page-locked host memory the device can address");
    }
    g->pop_sink = (double *)dev;
    g->pop_ring = ring_steps;
    return ML_OK;
}

ml_status ml_get_molecules(ml_grid *g, int what, double *dst, int dst_on_device, void *stream) {
    if (!g || !dst) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (what < 0 || what > 4) return fail(ML_ERR_INVALID_ARG, "unknown molecule quantity");
    if (g->nmol == 0) return ML_OK;
    cudaStream_t s = (cudaStream_t)stream;
    size_t n = what == 0 ? 2 * (size_t)g->pool
                         : (what == 3 ? (size_t)g->nmol : (what == 4 ? (size_t)g->nmol * MAXLEV : 3 * (size_t)g->nmol));
    if (dst_on_device < 0 || dst_on_device > 2) return fail(ML_ERR_INVALID_ARG, "dst_on_device must be 0, 1 or 2");
    double *tgt = dst_on_device == 1 ? dst : g->d_export;
    cudaError_t e = g->prec ? launch_mol_export<double>(what, g->nmol, g->d_nlev, g->d_off, (const cx<double> *)g->d_rho,
                                                        (const double *)g->d_Et, (const double *)g->d_mudot, g->d_energy,
                                                        g->pool, tgt, s)
                            : launch_mol_export<float>(what, g->nmol, g->d_nlev, g->d_off, (const cx<float> *)g->d_rho,
                                                       (const float *)g->d_Et, (const float *)g->d_mudot, g->d_energy,
                                                       g->pool, tgt, s);
    CK(e);
    if (dst_on_device != 1) {
        CK(cudaMemcpyAsync(dst, g->d_export, n * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (dst_on_device == 0) CK(cudaStreamSynchronize(s));
    }
    return ML_OK;
}

ml_status ml_flux(ml_grid *g, int id, double *out, void *stream) {
    if (!g || !out) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (id < 0 || id >= (int)g->planes.size()) return fail(ML_ERR_INVALID_ARG, "no such plane");
    cudaStream_t s = (cudaStream_t)stream;
    ml_status st = g->prec ? fold_planes<double>(g, s) : fold_planes<float>(g, s);
    if (st != ML_OK) return st;
    Plane &p = g->planes[id];
    CK(launch_flux_reduce(p.d_acc, p.nb * p.nc, p.nfreq, g->d_fpart, g->d_scalar, s));
    CK(cudaMemcpyAsync(out, g->d_scalar, p.nfreq * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ML_OK;
}

ml_status ml_flux_data(ml_grid *g, int id, double *out, void *stream) {
    if (!g || !out) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (id < 0 || id >= (int)g->planes.size()) return fail(ML_ERR_INVALID_ARG, "no such plane");
    cudaStream_t s = (cudaStream_t)stream;
    ml_status st = g->prec ? fold_planes<double>(g, s) : fold_planes<float>(g, s);
    if (st != ML_OK) return st;
    Plane &p = g->planes[id];
    CK(cudaMemcpyAsync(out, p.d_acc, 4 * (size_t)p.nfreq * p.nb * p.nc * sizeof(double2), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ML_OK;
}

ml_status ml_absorbed(ml_grid *g, double *out, void *stream) {
    if (!g || !out) return fail(ML_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_sum_doubles(g->absorbed_part, g->nblocks, g->d_scalar, s));
    CK(cudaMemcpyAsync(out, g->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ML_OK;
}

ml_status ml_sync_status(ml_grid *g, void *stream) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    int st = 0;
    CK(cudaMemcpy(&st, g->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemset(g->d_status, 0, sizeof(int)));
    if (st == ML_ERR_NUMERIC) return fail(ML_ERR_NUMERIC, "non-finite molecular field or current");
    if (st == ML_ERR_TIMEOUT) return fail(ML_ERR_TIMEOUT, "device wait timed out");
    if (st != 0) return fail((ml_status)st, "device status " + std::to_string(st));
    return ML_OK;
}

ml_status ml_set_wait_limit(ml_grid *g, int64_t probes) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    if (probes < 0 || probes > 0x7fffffffll) return fail(ML_ERR_INVALID_ARG, "probes must be in 0 .. 2^31 - 1");
    g->wait_limit = (uint32_t)probes;
    return ML_OK;
}

int64_t ml_step_count(const ml_grid *g) { return g ? g->step : -1; }
int64_t ml_launch_count(const ml_grid *g) { return g ? g->launches : -1; }

ml_status ml_set_timing(ml_grid *g, int enable) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    g->timing = enable != 0;
    return ML_OK;
}

ml_status ml_timing(ml_grid *g, double *ms, int64_t *counts) {
    if (!g) return fail(ML_ERR_INVALID_ARG, "null grid");
    double t[6] = {0, 0, 0, 0, 0, 0};
    int64_t c[6] = {0, 0, 0, 0, 0, 0};
    for (auto &x : g->timed) {
        CK(cudaEventSynchronize(x.b));
        float f = 0.f;
        CK(cudaEventElapsedTime(&f, x.a, x.b));
        t[x.kind] += f;
        c[x.kind]++;
        g->ev_free.push_back(x.a);
        g->ev_free.push_back(x.b);
    }
    g->timed.clear();
    for (int q = 0; q < 6; q++) {
        if (ms) ms[q] = t[q];
        if (counts) counts[q] = c[q];
    }
    return ML_OK;
}
int ml_molecule_count(const ml_grid *g) { return g ? g->nmol : -1; }

// ------------------------------------------------------------------ checkpoint

std::vector<Blob> ml::state_blobs(ml_grid *g) {
    std::vector<Blob> b;
    for (int c = 0; c < 6; c++) b.push_back({g->F[g->cur][c], g->vol * g->esz});
    for (int a = 0; a < 3; a++)
        for (int q = 0; q < 2; q++)
            if (g->psi_n[a]) {
                b.push_back({g->psiH[g->cur][a][q], g->psi_n[a] * g->esz});
                b.push_back({g->psiE[a][q], g->psi_n[a] * g->esz});
            }
    if (g->JD) b.push_back({g->JD, 3 * (size_t)g->npole * g->jcnt * g->esz});
    if (g->PD) b.push_back({g->PD, 3 * (size_t)g->npole * g->jcnt * g->esz});
    b.push_back({g->absorbed_part, (size_t)g->nblocks * sizeof(double)});
    if (g->nmol) {
        b.push_back({g->d_rho, 2 * (size_t)g->pool * g->esz});
        b.push_back({g->d_energy, (size_t)g->nmol * sizeof(double)});
        b.push_back({g->d_Et, 3 * (size_t)g->nmol * g->esz});
        b.push_back({g->d_mudot, 3 * (size_t)g->nmol * g->esz});
        b.push_back({g->d_c, 3 * (size_t)g->nmol * g->esz});
    }
    for (auto &p : g->planes) {
        size_t ncell = (size_t)p.nb * p.nc;
        b.push_back({p.d_acc, 4 * (size_t)p.nfreq * ncell * sizeof(double2)});
        b.push_back({p.d_buf, (size_t)DFT_KMAX * 4 * ncell * g->esz});
    }
    return b;
}

namespace {
const uint64_t kMagic = 0x4d4c434b50543031ull;  // "MLCKPT01"
}  // namespace

ml_status ml_checkpoint(ml_grid *g, void *host_buf, size_t *bytes, void *stream) {
    if (!g || !bytes) return fail(ML_ERR_INVALID_ARG, "null argument");
    auto blobs = state_blobs(g);
    size_t need = 4 * sizeof(uint64_t);
    for (auto &b : blobs) need += b.bytes;
    if (!host_buf) {
        *bytes = need;
        return ML_OK;
    }
    if (*bytes < need) return fail(ML_ERR_INVALID_ARG, "checkpoint buffer too small");
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t *hdr = (uint64_t *)host_buf;
    hdr[0] = kMagic;
    hdr[1] = (uint64_t)g->step;
    hdr[2] = (uint64_t)g->nsamp;
    hdr[3] = (uint64_t)g->samp_step0;
    char *o = (char *)host_buf + 4 * sizeof(uint64_t);
    for (auto &b : blobs) {
        CK(cudaMemcpyAsync(o, b.p, b.bytes, cudaMemcpyDeviceToHost, s));
        o += b.bytes;
    }
    CK(cudaStreamSynchronize(s));
    *bytes = need;
    return ML_OK;
}

ml_status ml_restore(ml_grid *g, const void *host_buf, size_t bytes, void *stream) {
    if (!g || !host_buf) return fail(ML_ERR_INVALID_ARG, "null argument");
    auto blobs = state_blobs(g);
    size_t need = 4 * sizeof(uint64_t);
    for (auto &b : blobs) need += b.bytes;
    const uint64_t *hdr = (const uint64_t *)host_buf;
    if (bytes != need || hdr[0] != kMagic) return fail(ML_ERR_INVALID_ARG, "checkpoint does not match this grid");
    cudaStream_t s = (cudaStream_t)stream;
    const char *o = (const char *)host_buf + 4 * sizeof(uint64_t);
    for (auto &b : blobs) {
        CK(cudaMemcpyAsync(b.p, o, b.bytes, cudaMemcpyHostToDevice, s));
        o += b.bytes;
    }
    CK(cudaStreamSynchronize(s));
    g->step = (long long)hdr[1];
    g->nsamp = (int)hdr[2];
    g->samp_step0 = (long long)hdr[3];
    return ML_OK;
}
