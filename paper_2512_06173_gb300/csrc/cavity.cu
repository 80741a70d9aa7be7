// Single-mode cavity solver (Sec. II, "Classical photonic dynamics in normal modes"),
// in the single-mode limit the paper implements: one mode of frequency w_c per
// polarisation lambda = x, y with mode function e_lambda / sqrt(V).
//
// Every molecule m sees E~_m = gamma_m Eu (Eq. E_normalmode; Eu is kept on the device)
// and advances rho exactly as in ml_step.  The new dipole sum d^{n+1} (Eq. dklambda_def)
// is added in a fixed order; then q and p advance by velocity Verlet on
// q'' = -w_c^2 q - eps d (Eq. eom_cavmd_a) with half kicks at d^n and d^{n+1}, and the
// next field is Eu = -(eps q + eps^2 / w_c^2 d).  Per step, on the caller's stream:
//   - ensembles of two-level molecules: one launch (molecule_cavity_kernel): per-block
//     partial sums, and the block that takes the last ticket adds them and steps the mode;
//   - other ensembles: the warp-per-molecule uniform-field kernel writes gamma_m <mu>
//     per molecule, then cavity_mode_kernel: CAV_NB blocks add them in a fixed order
//     into one FP64 partial each, and the last block (a ticket counter) adds the
//     partials by a fixed tree and steps the mode.
// Nothing waits on another block: the last block is whichever takes the final ticket.
// Runs of 64 steps are captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "grid.cuh"

using namespace ml;

namespace {

constexpr int CAV_NB = 128;   // blocks of the dipole sum
constexpr int CAV_NT = 256;   // threads per block
constexpr int MODE_N = 9;     // q_x q_y p_x p_y d_x d_y Eu_x Eu_y Eu_z
constexpr int CAV_SEQ = 64;   // steps per captured sequence
static_assert(CAV_NB <= CAV_NT, "the last block loads one partial per thread");

template <typename T>
__global__ void __launch_bounds__(CAV_NT) cavity_mode_kernel(const T *gmu, long long M, double *part, unsigned *ticket,
                                                             double *mode, float *euf, double wc, double eps, double dt) {
    __shared__ double red[3][CAV_NT];
    __shared__ bool last;
    const int tid = threadIdx.x;
    double s[3] = {0.0, 0.0, 0.0};
    for (long long m = (long long)blockIdx.x * CAV_NT + tid; m < M; m += (long long)CAV_NB * CAV_NT)
        for (int c = 0; c < 3; c++) s[c] += (double)gmu[3 * m + c];
    for (int c = 0; c < 3; c++) red[c][tid] = s[c];
    __syncthreads();
    for (int o = CAV_NT / 2; o > 0; o >>= 1) {
        if (tid < o)
            for (int c = 0; c < 3; c++) red[c][tid] += red[c][tid + o];
        __syncthreads();
    }
    if (tid == 0) {
        for (int c = 0; c < 3; c++) part[3 * blockIdx.x + c] = red[c][0];
        __threadfence();  // the partial is visible before the ticket is taken
        last = atomicAdd(ticket, 1u) == CAV_NB - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: the CAV_NB partials by the same fixed tree
    __threadfence();
    for (int l = 0; l < 2; l++) red[l][tid] = tid < CAV_NB ? __ldcg(part + 3 * tid + l) : 0.0;
    __syncthreads();
    for (int o = CAV_NT / 2; o > 0; o >>= 1) {
        if (tid < o)
            for (int l = 0; l < 2; l++) red[l][tid] += red[l][tid + o];
        __syncthreads();
    }
    if (tid != 0) return;
    const double d[2] = {red[0][0], red[1][0]};
    cavity_advance_mode(mode, euf, d, wc, eps, dt);
    *ticket = 0u;  // ready for the next launch
}

}  // namespace

struct ml_cavity {
    int prec = 0;
    size_t esz = 4;
    int M = 0;
    long long pool = 0;
    double dt = 0.0, wc = 0.0, eps = 0.0;
    bool two_level = true;
    bool exact_only = true;  // every molecule is kind 0 (the exact 2x2 step)
    int mu_zero = 7;         // bit c: mu_c is zero for every molecule
    long long step = 0;
    int *d_nlev = nullptr, *d_kind = nullptr, *d_nsub = nullptr, *d_cmask = nullptr, *d_status = nullptr;
    long long *d_off = nullptr;
    void *d_gamma = nullptr, *d_decay = nullptr, *d_deph = nullptr, *d_H0 = nullptr, *d_mu = nullptr,
         *d_rho = nullptr, *d_Et = nullptr, *d_mudot = nullptr, *d_c = nullptr, *d_gmu = nullptr;
    double *d_energy = nullptr, *d_mode = nullptr, *d_part = nullptr, *d_export = nullptr;
    double *d_bpart = nullptr;  // two-level molecules: per-block dipole sums of the molecule kernel
    float *d_euf = nullptr;     // FP32 molecules: the mode's field Eu in FP32
    unsigned *d_ticket = nullptr;
    std::vector<ml::DevBuf> allocs;
    // CAV_SEQ steps captured once into a graph (the arguments never change) and replayed
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

ml_status cav_alloc(ml_cavity *c, void **p, size_t bytes) {
    return dev_alloc(c->allocs, p, std::max<size_t>(bytes, 16));
}

template <typename V>
ml_status cav_upload(ml_cavity *c, V **dst, const std::vector<V> &v) {
    ml_status s = cav_alloc(c, (void **)dst, v.size() * sizeof(V));
    if (s != ML_OK) return s;
    if (!v.empty()) CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice));
    return ML_OK;
}

// doubles, stored in the molecules' precision
ml_status cav_upload_reals(ml_cavity *c, void **dst, const std::vector<double> &v) {
    if (c->prec) return cav_upload(c, (double **)dst, v);
    std::vector<float> f(v.begin(), v.end());
    return cav_upload(c, (float **)dst, f);
}

template <typename T>
void fill_cavity_args(ml_cavity *c, MolArgs<T> &m) {
    m = MolArgs<T>{};
    m.nmol = c->M;
    m.dt = (T)c->dt;
    m.nlev = c->d_nlev; m.off = c->d_off; m.kind = c->d_kind; m.nsub = c->d_nsub; m.cmask = c->d_cmask;
    m.gamma = (const T *)c->d_gamma; m.decay = (const T *)c->d_decay; m.dephase = (const T *)c->d_deph;
    m.H0 = (const cx<T> *)c->d_H0; m.mu = (const cx<T> *)c->d_mu; m.pool = c->pool;
    m.rho = (cx<T> *)c->d_rho;
    m.Et = (T *)c->d_Et; m.mudot = (T *)c->d_mudot; m.c = (T *)c->d_c;
    m.energy = c->d_energy; m.status = c->d_status;
    m.two_level = c->two_level ? 1 : 0;
    m.exact_only = c->exact_only ? 1 : 0;
    m.mu_zero = c->mu_zero;
    m.Eu = (const T *)(const void *)(sizeof(T) == 8 ? (c->d_mode ? c->d_mode + 6 : nullptr) : (const void *)c->d_euf);
    m.gmu = (T *)c->d_gmu;
    m.dpart = c->d_bpart;
    m.mode = c->d_mode;
    m.euf = c->d_euf;
    m.ticket = c->d_ticket;
    m.wc = c->wc;
    m.eps = c->eps;
    m.mdt = c->dt;
}

template <typename T>
ml_status enqueue_steps(ml_cavity *c, long long nsteps, cudaStream_t s) {
    MolArgs<T> m;
    fill_cavity_args<T>(c, m);
    for (long long it = 0; it < nsteps; it++) {
        if (c->two_level) {
            // one launch: the molecules' partial sums and, in its last block, the mode step
            CK(launch_molecules_cavity<T>(m, s));
            continue;
        }
        CK(launch_molecules_uniform<T>(m, s));
        cavity_mode_kernel<T><<<CAV_NB, CAV_NT, 0, s>>>((const T *)c->d_gmu, c->M, c->d_part, c->d_ticket, c->d_mode,
                                                         c->d_euf, c->wc, c->eps, c->dt);
        CK(cudaGetLastError());
    }
    return ML_OK;
}

template <typename T>
ml_status cavity_steps(ml_cavity *c, long long nsteps, cudaStream_t s) {
    const long long reps = nsteps / CAV_SEQ;
    if (reps > 0 && !c->exec) {
        if (!c->cap) CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        const ml_status e = enqueue_steps<T>(c, CAV_SEQ, c->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(c->cap, &graph);
        if (e != ML_OK) {
            if (graph) cudaGraphDestroy(graph);
            return e;
        }
        CK(ce);
        c->graph = graph;
        CK(cudaGraphInstantiate(&c->exec, c->graph, 0));
    }
    for (long long r = 0; r < reps; r++) {
        CK(cudaGraphLaunch(c->exec, s));
        c->step += CAV_SEQ;
    }
    const long long rest = nsteps - reps * CAV_SEQ;
    ml_status st = enqueue_steps<T>(c, rest, s);
    if (st != ML_OK) return st;
    c->step += rest;
    return ML_OK;
}

}  // namespace

namespace {

// Validate and copy a molecule table into `c` (precision already set): device arrays of
// the molecule step, the work arrays, and FP64 d0 = sum_m gamma_m <mu_x,y>(rho0).
ml_status load_ensemble(ml_cavity *c, const ml_molecule_desc *md, double (&d0)[2]) {
    if (md->count < 1) return fail(ML_ERR_INVALID_ARG, "an ensemble needs at least one molecule");
    if (!md->nlev || !md->off || !md->gamma || !md->decay || !md->dephase || !md->kind || !md->nsub || !md->H0 ||
        !md->mu || !md->rho)
        return fail(ML_ERR_INVALID_ARG, "null molecule array");
    const int M = md->count;
    std::vector<int> nlev(M), kind(M), nsub(M), cmask(M);
    std::vector<long long> off(M);
    std::vector<double> gamma(M), decay(M), deph(M), H0, rho, mu;
    long long pool = 0;
    for (int m = 0; m < M; m++) {
        const int n = md->nlev[m];
        if (n < 2 || n > ML_MAX_LEVELS) return fail(ML_ERR_INVALID_ARG, "nlev must be 2..8");
        if (md->off[m] < 0 || md->off[m] + (long long)n * n > md->pool) return fail(ML_ERR_INVALID_ARG, "pool offset out of range");
        if (md->kind[m] != 0 && md->kind[m] != 1) return fail(ML_ERR_INVALID_ARG, "kind must be 0 or 1");
        if (md->kind[m] == 0 && (n != 2 || md->decay[m] != 0.0 || md->dephase[m] != 0.0))
            return fail(ML_ERR_INVALID_ARG, "kind 0 needs two levels and no Lindblad terms");
        if (md->nsub[m] < 1) return fail(ML_ERR_INVALID_ARG, "nsub must be >= 1");
        if (md->decay[m] < 0.0 || md->dephase[m] < 0.0) return fail(ML_ERR_INVALID_ARG, "negative rate");
        if (!std::isfinite(md->gamma[m])) return fail(ML_ERR_INVALID_ARG, "non-finite gamma");
        nlev[m] = n;
        kind[m] = md->kind[m];
        nsub[m] = md->nsub[m];
        gamma[m] = md->gamma[m];
        decay[m] = md->decay[m];
        deph[m] = md->dephase[m];
        off[m] = pool;
        pool += (long long)n * n;
    }
    H0.resize(2 * pool);
    rho.resize(2 * pool);
    mu.assign(2 * 3 * pool, 0.0);
    d0[0] = d0[1] = 0.0;
    for (int m = 0; m < M; m++) {
        const int nn = nlev[m] * nlev[m];
        int cm = 0;
        for (int e = 0; e < nn; e++) {
            const long long src = md->off[m] + e, dst = off[m] + e;
            H0[2 * dst] = md->H0[2 * src];
            H0[2 * dst + 1] = md->H0[2 * src + 1];
            rho[2 * dst] = md->rho[2 * src];
            rho[2 * dst + 1] = md->rho[2 * src + 1];
            for (int c = 0; c < 3; c++) {
                const double re = md->mu[2 * (c * md->pool + src)], im = md->mu[2 * (c * md->pool + src) + 1];
                mu[2 * (c * pool + dst)] = re;
                mu[2 * (c * pool + dst) + 1] = im;
                if (re != 0.0 || im != 0.0) cm |= 1 << c;
                // <mu_c> = Re Tr(rho mu_c) = sum_e Re(rho_e conj(mu_c,e)) for Hermitian mu_c
                if (c < 2) d0[c] += gamma[m] * (rho[2 * dst] * re + rho[2 * dst + 1] * im);
            }
        }
        cmask[m] = cm;
    }
    c->esz = c->prec ? 8 : 4;
    c->M = M;
    c->pool = pool;
    c->two_level = true;
    c->exact_only = true;
    c->mu_zero = 7;
    for (int m = 0; m < M; m++) {
        c->two_level = c->two_level && nlev[m] == 2;
        c->exact_only = c->exact_only && kind[m] == 0;
        c->mu_zero &= ~cmask[m];
    }
    ml_status st;
#define CAV(x)                \
    do {                      \
        st = (x);             \
        if (st != ML_OK) return st; \
    } while (0)
    CAV(cav_upload(c, &c->d_nlev, nlev));
    CAV(cav_upload(c, &c->d_kind, kind));
    CAV(cav_upload(c, &c->d_nsub, nsub));
    CAV(cav_upload(c, &c->d_cmask, cmask));
    CAV(cav_upload(c, &c->d_off, off));
    CAV(cav_upload_reals(c, &c->d_gamma, gamma));
    CAV(cav_upload_reals(c, &c->d_decay, decay));
    CAV(cav_upload_reals(c, &c->d_deph, deph));
    CAV(cav_upload_reals(c, &c->d_H0, H0));
    CAV(cav_upload_reals(c, &c->d_mu, mu));
    CAV(cav_upload_reals(c, &c->d_rho, rho));
    CAV(cav_alloc(c, &c->d_Et, 3 * (size_t)M * c->esz));
    CAV(cav_alloc(c, &c->d_mudot, 3 * (size_t)M * c->esz));
    CAV(cav_alloc(c, &c->d_c, 3 * (size_t)M * c->esz));
    CAV(cav_alloc(c, &c->d_gmu, 3 * (size_t)M * c->esz));
    CAV(cav_upload(c, &c->d_energy, std::vector<double>(M, 0.0)));
    CAV(cav_upload(c, &c->d_status, std::vector<int>(1, 0)));
    CAV(cav_upload(c, &c->d_ticket, std::vector<unsigned>(1, 0u)));
    CAV(cav_alloc(c, (void **)&c->d_part, 3 * CAV_NB * sizeof(double)));
    CAV(cav_alloc(c, (void **)&c->d_bpart, 3 * (size_t)((M + MU_THREADS_HOST - 1) / MU_THREADS_HOST) * sizeof(double)));
    CAV(cav_alloc(c, (void **)&c->d_export,
                  std::max<size_t>((size_t)std::max<long long>(2 * pool, (long long)M * MAXLEV), 1) * sizeof(double)));
#undef CAV
    return ML_OK;
}

}  // namespace

ml_status ml_cavity_create(const ml_cavity_desc *d, const ml_molecule_desc *md, ml_cavity **out) {
    if (!d || !md || !out) return fail(ML_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(d->omega_c > 0.0) || !std::isfinite(d->omega_c)) return fail(ML_ERR_INVALID_ARG, "omega_c must be > 0");
    if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(ML_ERR_INVALID_ARG, "dt must be > 0");
    if (!std::isfinite(d->coupling)) return fail(ML_ERR_INVALID_ARG, "non-finite coupling");
    for (int l = 0; l < 2; l++)
        if (!std::isfinite(d->q0[l]) || !std::isfinite(d->p0[l])) return fail(ML_ERR_INVALID_ARG, "non-finite mode state");
    if (d->precision != ML_F32 && d->precision != ML_F64) return fail(ML_ERR_INVALID_ARG, "precision must be ML_F32 or ML_F64");
    ml_cavity *c = new ml_cavity();
    c->prec = d->precision;
    c->dt = d->dt;
    c->wc = d->omega_c;
    c->eps = d->coupling;
    double d0[2];
    ml_status st = load_ensemble(c, md, d0);
    if (st == ML_OK) {
        std::vector<double> mode(MODE_N, 0.0);
        for (int l = 0; l < 2; l++) {
            mode[l] = d->q0[l];
            mode[2 + l] = d->p0[l];
            mode[4 + l] = d0[l];
            mode[6 + l] = -(c->eps * d->q0[l] + c->eps * c->eps / (c->wc * c->wc) * d0[l]);
        }
        st = cav_upload(c, &c->d_mode, mode);
        if (st == ML_OK && !c->prec) st = cav_upload(c, &c->d_euf, std::vector<float>(mode.begin() + 6, mode.end()));
    }
    if (st != ML_OK) {
        ml_cavity_destroy(c);
        return st;
    }
    *out = c;
    return ML_OK;
}

ml_status ml_cavity_destroy(ml_cavity *c) {
    if (!c) return ML_OK;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->cap) cudaStreamDestroy(c->cap);
    cudaDeviceSynchronize();
    dev_free_all(c->allocs);
    delete c;
    return ML_OK;
}

ml_status ml_cavity_step(ml_cavity *c, int64_t nsteps, void *stream) {
    if (!c) return fail(ML_ERR_INVALID_ARG, "null cavity");
    if (nsteps < 0) return fail(ML_ERR_INVALID_ARG, "negative step count");
    cudaStream_t s = (cudaStream_t)stream;
    return c->prec ? cavity_steps<double>(c, nsteps, s) : cavity_steps<float>(c, nsteps, s);
}

ml_status ml_cavity_mode(ml_cavity *c, double *out, void *stream) {
    if (!c || !out) return fail(ML_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    double buf[MODE_N];
    int status = 0;
    CK(cudaMemcpyAsync(buf, c->d_mode, sizeof(buf), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < 6; q++) out[q] = buf[q];
    if (status) return fail(ML_ERR_NUMERIC, "a molecule's field or dipole rate became non-finite");
    return ML_OK;
}

ml_status ml_cavity_get_molecules(ml_cavity *c, int what, double *dst, void *stream) {
    if (!c || !dst) return fail(ML_ERR_INVALID_ARG, "null argument");
    if (what < ML_MOL_RHO || what > ML_MOL_POP) return fail(ML_ERR_INVALID_ARG, "unknown molecular quantity");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = what == ML_MOL_RHO ? 2 * (size_t)c->pool
                                        : (what == ML_MOL_ENERGY ? (size_t)c->M
                                                                 : (what == ML_MOL_POP ? (size_t)c->M * MAXLEV : 3 * (size_t)c->M));
    cudaError_t e = c->prec ? launch_mol_export<double>(what, c->M, c->d_nlev, c->d_off, (const cx<double> *)c->d_rho,
                                                        (const double *)c->d_Et, (const double *)c->d_mudot,
                                                        c->d_energy, c->pool, c->d_export, s)
                            : launch_mol_export<float>(what, c->M, c->d_nlev, c->d_off, (const cx<float> *)c->d_rho,
                                                       (const float *)c->d_Et, (const float *)c->d_mudot,
                                                       c->d_energy, c->pool, c->d_export, s);
    CK(e);
    CK(cudaMemcpyAsync(dst, c->d_export, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ML_OK;
}

int64_t ml_cavity_step_count(const ml_cavity *c) { return c ? c->step : -1; }

// ---- Laser-driven molecules (classical path, Eq. E_analytical) ----------------------
// The molecules of an ml_cavity shell without the mode: every step is one launch of
// the uniform-field molecule kernel with the laser's plane wave; the absolute step of a
// launch is a device counter (advanced by a tick after each run of steps) plus the
// launch's offset in that run, so that 64-step runs can be replayed from a graph.

struct ml_drive {
    ml_cavity *c = nullptr;
    double E0 = 0.0, k = 0.0, phase = 0.0, xi0 = 0.0, W = 0.0, pol[3] = {0.0, 0.0, 0.0}, dt = 0.0;
    double *d_z = nullptr;        // FP64 molecules: z_m
    float2 *d_zr = nullptr;       // FP32 molecules: z_m - xi0 as a float pair
    float2 *d_tt = nullptr;       // FP32 molecules: t of each launch of the next run as a float pair
    long long *d_base = nullptr;
    long long step = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// a double as a float pair: hi = the nearest float, lo = the remainder rounded
__host__ __device__ inline float2 split_pair(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// After a run of n launches: advance the run's first step and write, for each launch q
// of the next run, t = (first step + q) dt as a float pair (FP64 here, once per run).
__global__ void drive_tick_kernel(long long *base, int n, float2 *tt, double dt) {
    const long long b = *base + n;
    __syncthreads();  // every thread has read the old value
    if (threadIdx.x == 0) *base = b;
    tt[threadIdx.x] = split_pair((double)(b + threadIdx.x) * dt);
}

template <typename T>
ml_status enqueue_drive(ml_drive *d, int nsteps, cudaStream_t s) {
    if (nsteps <= 0) return ML_OK;
    MolArgs<T> m;
    fill_cavity_args<T>(d->c, m);
    m.dpart = nullptr;
    m.laser = 1;
    m.zpos = d->d_z;
    m.lbase = d->d_base;
    m.ldt = d->dt;
    m.lxi0 = d->xi0;
    m.lzr = d->d_zr;
    m.ltt = d->d_tt;
    m.lk = (T)d->k;
    m.lphase = (T)d->phase;
    m.lW = (T)d->W;
    m.lE0 = (T)d->E0;
    for (int c = 0; c < 3; c++) m.lpol[c] = (T)d->pol[c];
    for (int q = 0; q < nsteps; q++) {
        m.lstep = q;
        CK(launch_molecules_uniform<T>(m, s));
    }
    if (sizeof(T) == 8) {
        CK(launch_tick(d->d_base, nsteps, s));
    } else {
        drive_tick_kernel<<<1, CAV_SEQ, 0, s>>>(d->d_base, nsteps, d->d_tt, d->dt);
        CK(cudaGetLastError());
    }
    return ML_OK;
}

template <typename T>
ml_status drive_steps(ml_drive *d, long long nsteps, cudaStream_t s) {
    const long long reps = nsteps / CAV_SEQ;
    if (reps > 0 && !d->exec) {
        if (!d->cap) CK(cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal));
        const ml_status e = enqueue_drive<T>(d, CAV_SEQ, d->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(d->cap, &graph);
        if (e != ML_OK) {
            if (graph) cudaGraphDestroy(graph);
            return e;
        }
        CK(ce);
        d->graph = graph;
        CK(cudaGraphInstantiate(&d->exec, d->graph, 0));
    }
    for (long long r = 0; r < reps; r++) {
        CK(cudaGraphLaunch(d->exec, s));
        d->step += CAV_SEQ;
        d->c->step += CAV_SEQ;
    }
    const int rest = (int)(nsteps - reps * CAV_SEQ);
    ml_status st = enqueue_drive<T>(d, rest, s);
    if (st != ML_OK) return st;
    d->step += rest;
    d->c->step += rest;
    return ML_OK;
}

}  // namespace

ml_status ml_drive_create(const ml_drive_desc *dd, const ml_molecule_desc *md, ml_drive **out) {
    if (!dd || !md || !out) return fail(ML_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (!(dd->dt > 0.0) || !std::isfinite(dd->dt)) return fail(ML_ERR_INVALID_ARG, "dt must be > 0");
    if (!(dd->half_width > 0.0) || !std::isfinite(dd->half_width)) return fail(ML_ERR_INVALID_ARG, "half_width must be > 0");
    if (!std::isfinite(dd->amplitude) || !std::isfinite(dd->omega) || !std::isfinite(dd->phase) ||
        !std::isfinite(dd->center))
        return fail(ML_ERR_INVALID_ARG, "non-finite pulse parameter");
    for (int c = 0; c < 3; c++)
        if (!std::isfinite(dd->polarization[c])) return fail(ML_ERR_INVALID_ARG, "non-finite polarisation");
    if (dd->precision != ML_F32 && dd->precision != ML_F64) return fail(ML_ERR_INVALID_ARG, "precision must be ML_F32 or ML_F64");
    if (md->count >= 1 && !md->pos) return fail(ML_ERR_INVALID_ARG, "null molecule positions");
    ml_drive *d = new ml_drive();
    d->c = new ml_cavity();
    d->c->prec = dd->precision;
    d->c->dt = dd->dt;
    d->E0 = dd->amplitude;
    d->k = dd->omega;
    d->phase = dd->phase;
    d->xi0 = dd->center;
    d->W = dd->half_width;
    d->dt = dd->dt;
    for (int c = 0; c < 3; c++) d->pol[c] = dd->polarization[c];
    double d0[2];
    ml_status st = load_ensemble(d->c, md, d0);
    if (st == ML_OK) {
        std::vector<double> z(md->count);
        for (int m = 0; m < md->count; m++) {
            z[m] = md->pos[3 * m + 2];
            if (!std::isfinite(z[m])) st = fail(ML_ERR_INVALID_ARG, "non-finite position");
        }
        if (st == ML_OK && d->c->prec) st = cav_upload(d->c, &d->d_z, z);
        if (st == ML_OK && !d->c->prec) {
            std::vector<float2> zr(md->count), tt(CAV_SEQ);
            for (int m = 0; m < md->count; m++) zr[m] = split_pair(z[m] - d->xi0);
            for (int q = 0; q < CAV_SEQ; q++) tt[q] = split_pair((double)q * d->dt);
            st = cav_upload(d->c, &d->d_zr, zr);
            if (st == ML_OK) st = cav_upload(d->c, &d->d_tt, tt);
        }
        if (st == ML_OK) st = cav_upload(d->c, &d->d_base, std::vector<long long>(1, 0));
    }
    if (st != ML_OK) {
        ml_drive_destroy(d);
        return st;
    }
    *out = d;
    return ML_OK;
}

ml_status ml_drive_destroy(ml_drive *d) {
    if (!d) return ML_OK;
    if (d->exec) cudaGraphExecDestroy(d->exec);
    if (d->graph) cudaGraphDestroy(d->graph);
    if (d->cap) cudaStreamDestroy(d->cap);
    ml_cavity_destroy(d->c);
    delete d;
    return ML_OK;
}

ml_status ml_drive_step(ml_drive *d, int64_t nsteps, void *stream) {
    if (!d) return fail(ML_ERR_INVALID_ARG, "null drive");
    if (nsteps < 0) return fail(ML_ERR_INVALID_ARG, "negative step count");
    cudaStream_t s = (cudaStream_t)stream;
    return d->c->prec ? drive_steps<double>(d, nsteps, s) : drive_steps<float>(d, nsteps, s);
}

ml_status ml_drive_get_molecules(ml_drive *d, int what, double *dst, void *stream) {
    if (!d) return fail(ML_ERR_INVALID_ARG, "null drive");
    ml_status st = ml_cavity_get_molecules(d->c, what, dst, stream);
    if (st != ML_OK) return st;
    int status = 0;
    CK(cudaMemcpy(&status, d->c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status) return fail(ML_ERR_NUMERIC, "a molecule's field or dipole rate became non-finite");
    return ML_OK;
}

int64_t ml_drive_step_count(const ml_drive *d) { return d ? d->step : -1; }
