// Host-side state of a grid (the opaque ml_grid of maxlink.h) and the pieces of
// the step driver that more than one source file of the library uses.
#pragma once
#include <string>
#include <vector>

#include "devmem.cuh"
#include "maxlink.h"
#include "ml_internal.cuh"

namespace ml {

// Record `msg` for ml_last_error and return `s`.
inline ml_status fail(ml_status s, const std::string &msg) {
    set_last_error(msg);
    return s;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return ml::fail(ML_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

struct Plane {
    int axis, index, nfreq, nb, nc;
    std::vector<double> omega;
    double *d_omega = nullptr;
    void *d_ph = nullptr;  // e^{i w s dt}, s < DFT_KMAX, in the field type: [re: s x nfreq | im: s x nfreq]
    void *d_buf = nullptr;
    double2 *d_acc = nullptr;
};

}  // namespace ml

struct ml_grid {
    int prec = 0;
    size_t esz = 4;
    int nx = 0, ny = 0, nz = 0;
    double dt = 0.5;
    int per[3] = {0, 0, 0};
    int pml[6] = {0, 0, 0, 0, 0, 0};
    double pml_m = 3, smax = 3.2, kmax = 1, amax = 0.05;
    int ntx = 0, nty = 0, nchunk = 0, cz = 0, nblocks = 0;
    std::vector<int> zcut;  // chunk boundaries along z
    int *d_zcut = nullptr;
    uint8_t *d_tflags = nullptr;  // per tile: bit 0 = pole or design box, bit 1 = material, bit 2 = source
    uint8_t *d_tmode = nullptr;   // per tile: the field-pass body it takes
    int bodies = ml::YEE_BODIES_ALL;  // the field-pass kernel's body set (YEE_BODIES_*)
    int px = 0, py = 0;
    long long plane = 0;
    size_t vol = 0;  // padded elements per array
    void *F[2][6] = {};
    int cur = 0;
    void *cpml[3] = {};
    void *psiH[2][3][2] = {};
    void *psiE[3][2] = {};
    size_t psi_n[3] = {0, 0, 0};
    uint8_t *mat = nullptr;
    void *mat_cb = nullptr, *mat_dk = nullptr, *mat_db = nullptr, *mat_dp = nullptr;
    int dbox[6] = {0, 0, 0, 0, 0, 0};
    void *dcb = nullptr;
    int jbox[6] = {0, 0, 0, 0, 0, 0};
    int npole = 0;        // pole slots in use
    size_t jcnt = 0;      // cells of the pole box
    void *JD = nullptr;   // pole currents [slot][component][jcnt] over the pole box
    void *PD = nullptr;   // pole polarisations, same layout (null: no Lorentz pole)
    double *absorbed_part = nullptr;
    double *d_scalar = nullptr;
    double *d_fpart = nullptr;  // flux reduction partials (ML_MAX_FREQS x FLUX_NB)
    std::vector<ml::SrcDev> src;
    // molecules: host mirror of the static description
    int nmol = 0;
    long long pool = 0;
    std::vector<int> nlev, kind, nsub, cmask, win, wf, wraw;
    bool two_level = true;  // every molecule has two levels (pool offset 4 m)
    int *d_order = nullptr;      // packed molecule kernel: molecules in work-item order
    int4 *d_items = nullptr;     //   and its work items (first, count, levels, kind | nsub << 4)
    int nitems = 0;
    double *pop_sink = nullptr;  // device address of the caller's page-locked population ring
    long long pop_ring = 0;
    bool pop_off = false;        // set while the adjoint sweeps step the grid

    std::vector<long long> off;
    std::vector<double> pos, sigma, gamma, decay, deph, H0, mu, rho0;
    // molecules: device
    int *d_nlev = nullptr, *d_kind = nullptr, *d_nsub = nullptr, *d_cmask = nullptr, *d_win = nullptr,
        *d_wf = nullptr, *d_wraw = nullptr;
    long long *d_off = nullptr;
    double *d_pos = nullptr, *d_sigma = nullptr, *d_energy = nullptr, *d_export = nullptr;
    void *d_gamma = nullptr, *d_decay = nullptr, *d_deph = nullptr, *d_H0 = nullptr, *d_mu = nullptr,
         *d_rho = nullptr, *d_w = nullptr, *d_Et = nullptr, *d_mudot = nullptr, *d_c = nullptr;
    // molecular current box and the entry lists of its blocks
    int jb0[3] = {0, 0, 0}, jbn[3] = {0, 0, 0};
    int jnbx = 0, jnby = 0, jnb = 0, gcmask = 0;
    int *d_joff = nullptr;
    int4 *d_jent = nullptr;
    unsigned char *d_jmask = nullptr;  // per entry: the current kernel's column groups its x window meets
    int *d_moff = nullptr, *d_mlist = nullptr;  // molecule -> its entries
    // field-pass blocks split by whether they touch the current box: the others
    // run while the gather -> molecules -> current chain runs on the side stream
    int *d_blA = nullptr, *d_blB = nullptr;
    int nblA = 0, nblB = 0;
    cudaStream_t side = nullptr;
    bool overlap = false;
    // the current kernel and the field pass start while the kernel before them still
    // runs (programmatic dependent launch; ML_PDL=0 turns it off)
    bool pdl = true;  // tuning (ML_OVERLAP=1): run the molecule chain beside the clear field blocks
    cudaEvent_t ev_join = nullptr, ev_box = nullptr;
    void *d_part = nullptr;                     // gather partials (entries, 3)
    void *d_J[3] = {};
    ml::TmapSet tm[2];
    std::vector<ml::Plane> planes;
    int nsamp = 0;
    long long samp_step0 = 0;
    void *scratch = nullptr;
    int *d_status = nullptr;
    uint32_t wait_limit = 2000;  // probes of a field-pass plane wait (ml_set_wait_limit)
    long long step = 0;
    // tracing: CUDA events around each launch of ml_step, per kernel class
    bool timing = false;
    std::vector<cudaEvent_t> ev_free;
    struct Timed { cudaEvent_t a, b; int kind; };  // kind: 0 molecules 1 field 2 sample 3 fold 4 current 5 gather
    std::vector<Timed> timed;
    long long launches = 0;
    std::vector<ml::DevBuf> allocs;       // grid lifetime
    std::vector<ml::DevBuf> mol_allocs;   // rebuilt when molecules are added
};

namespace ml {

inline cudaEvent_t take_event(ml_grid *g) {
    if (!g->ev_free.empty()) {
        cudaEvent_t e = g->ev_free.back();
        g->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket one kernel launch with events when tracing is on; count every launch.
struct LaunchScope {
    ml_grid *g;
    cudaStream_t s;
    int kind;
    cudaEvent_t a = nullptr;
    LaunchScope(ml_grid *g_, cudaStream_t s_, int kind_) : g(g_), s(s_), kind(kind_) {
        g->launches++;
        if (g->timing) {
            a = take_event(g);
            cudaEventRecord(a, s);
        }
    }
    ~LaunchScope() {
        if (a) {
            cudaEvent_t b = take_event(g);
            cudaEventRecord(b, s);
            g->timed.push_back({a, b, kind});
        }
    }
};

// One device buffer of the grid's dynamical state (what a checkpoint holds).
struct Blob {
    void *p;
    size_t bytes;
};
std::vector<Blob> state_blobs(ml_grid *g);

// Enqueue nsteps coupled steps (the body of ml_step).
template <typename T>
ml_status step_impl(ml_grid *g, long long nsteps, cudaStream_t s);

// Kernel arguments of one grid (level `cur` = the field level the step reads).
template <typename T> void fill_mol_args(ml_grid *g, int cur, MolArgs<T> &m);
template <typename T> void fill_gath_args(ml_grid *g, int cur, GathArgs<T> &ga);
template <typename T> void fill_cur_args(ml_grid *g, CurArgs<T> &ca);
template <typename T> void fill_yee_args(ml_grid *g, int cur, YeeArgs<T> &y);
template <typename T> ImgArgs<T> image_args(const ml_grid *g, int lev);

// Fold the pending plane samples into the FP64 DFT accumulators.
template <typename T>
ml_status fold_planes(ml_grid *g, cudaStream_t s);

}  // namespace ml
