// Batches: many independent grids (uneven sizes, uneven molecule counts and level
// numbers) advanced by the same launches.  Per step:
//   gather -> molecules -> current   (one launch each over every instance's blocks)
//   field pass                        (one persistent launch over every instance's tiles)
//   plane fold every DFT_KMAX steps   (one launch over every instance's planes)
// The per-instance kernel arguments live in device arrays, written once per
// ml_batch_step call.  A 64-step sequence (an even number of steps, whole fold periods)
// is captured once into a CUDA graph and replayed; a device step counter, advanced by a
// tick at the end of the sequence, gives the kernels the absolute step (source time,
// DFT phases).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "grid.cuh"

using namespace ml;

struct ml_batch {
    std::vector<ml_grid *> g;
    int prec = 0;
    int sms = 148;
    int blocks_per_sm = 0;  // field-pass grid: blocks_per_sm x SMs (0 = one block per work item)
    bool use_graph = true;
    // programmatic dependent launch of the current and field-pass kernels (ML_PDL=0: off)
    bool pdl = true;
    bool mol_two_level = true;  // every instance's molecules are all two-level
    int bodies = ml::YEE_BODIES_ALL;  // field-pass body set covering every instance
    // host copies of the argument arrays (kept alive: they are the source of async copies)
    std::vector<unsigned char> h_yargs, h_gargs, h_cargs, h_margs, h_fdesc;
    std::vector<TmapSet> h_maps;
    std::vector<int> h_lev0;
    std::vector<int2> h_ywork, h_gwork, h_mwork, h_fwork;
    // device arrays
    void *d_yargs = nullptr, *d_gargs = nullptr, *d_cargs = nullptr, *d_margs = nullptr, *d_fdesc = nullptr;
    TmapSet *d_maps = nullptr;
    int *d_lev0 = nullptr;
    int2 *d_ywork = nullptr, *d_gwork = nullptr, *d_mwork = nullptr, *d_fwork = nullptr;
    long long *d_boff = nullptr;
    size_t cap[11] = {};  // capacities (bytes) of the device arrays above
    // captured sequence
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> sig;  // what the graph baked in
    long long launches = 0;
    std::vector<ml::DevBuf> mem;  // the device arrays above
    // tracing (ml_batch_set_timing): events around each launch of steps taken without the
    // graph, per kernel class {molecules, field pass, -, fold, current}
    bool timing = false;
    struct Timed { cudaEvent_t a, b; int kind; };
    std::vector<Timed> timed;
};

namespace {

constexpr int SEQ = 64;  // steps per captured sequence: two time levels, whole fold periods
static_assert(SEQ % DFT_KMAX == 0 && SEQ % 2 == 0, "a sequence starts at a fold boundary and on level 0");

ml_status ensure(ml_batch *bt, void **p, size_t &cap, size_t bytes) {
    if (bytes <= cap && *p) return ML_OK;
    if (*p) dev_release(bt->mem, *p);
    *p = nullptr;
    cap = 0;
    const size_t b = std::max<size_t>(bytes, 256);
    ml_status st = dev_alloc(bt->mem, p, b);
    if (st != ML_OK) return st;
    cap = b;
    return ML_OK;
}

template <typename V>
ml_status upload(ml_batch *b, int slot, void **dptr, const std::vector<V> &h, cudaStream_t s) {
    ml_status st = ensure(b, dptr, b->cap[slot], h.size() * sizeof(V));
    if (st != ML_OK) return st;
    if (!h.empty()) CK(cudaMemcpyAsync(*dptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
    return ML_OK;
}

void drop_graph(ml_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->sig.clear();
}

// Build and upload the argument arrays and work lists for the grids' present state.
template <typename T>
ml_status prepare(ml_batch *b, cudaStream_t s) {
    const int n = (int)b->g.size();
    std::vector<YeeArgs<T>> ya(n);
    std::vector<GathArgs<T>> ga(2 * n);
    std::vector<CurArgs<T>> ca(n);
    std::vector<MolArgs<T>> ma(2 * n);
    std::vector<FoldDesc<T>> fd;
    b->h_maps.resize(2 * n);
    b->h_lev0.resize(n);
    b->h_ywork.clear();
    b->h_gwork.clear();
    b->h_mwork.clear();
    b->h_fwork.clear();
    b->mol_two_level = true;
    for (int i = 0; i < n; i++) {
        ml_grid *g = b->g[i];
        if (g->nmol > 0) b->mol_two_level = b->mol_two_level && g->two_level;
        fill_yee_args<T>(g, 0, ya[i]);
        ya[i].blist = nullptr;
        b->h_maps[2 * i] = g->tm[0];
        b->h_maps[2 * i + 1] = g->tm[1];
        b->h_lev0[i] = g->cur;
        for (int t = 0; t < g->nblocks; t++) b->h_ywork.push_back(make_int2(i, t));
        if (g->nmol > 0) {
            fill_gath_args<T>(g, 0, ga[2 * i]);
            fill_gath_args<T>(g, 1, ga[2 * i + 1]);
            fill_cur_args<T>(g, ca[i]);
            fill_mol_args<T>(g, 0, ma[2 * i]);
            fill_mol_args<T>(g, 1, ma[2 * i + 1]);
            ma[2 * i].pop_sink = ma[2 * i + 1].pop_sink = nullptr;  // batches write no sink
            for (int q = 0; q < g->jnb; q++) b->h_gwork.push_back(make_int2(i, q));
            if (g->nitems > 0)  // packed molecule items, four warps per block
                for (int it = 0; it < g->nitems; it += 4) b->h_mwork.push_back(make_int2(i, it));
            else
                for (int m0 = 0; m0 < g->nmol; m0 += 4) b->h_mwork.push_back(make_int2(i, m0));
        }
        for (auto &p : g->planes) {
            FoldDesc<T> d{};
            d.buf = (const T *)p.d_buf;
            d.ncell = p.nb * p.nc;
            d.nfreq = p.nfreq;
            d.omega = p.d_omega;
            d.ph = (const T *)p.d_ph;
            d.step_base = g->step;
            d.acc = p.d_acc;
            const int di = (int)fd.size();
            fd.push_back(d);
            const long long nent = 4ll * d.ncell;
            for (long long c = 0; c * 256 < nent; c++) b->h_fwork.push_back(make_int2(di, (int)c));
        }
    }
    auto bytes = [](auto &v) {
        std::vector<unsigned char> out(v.size() * sizeof(v[0]));
        if (!v.empty()) std::memcpy(out.data(), v.data(), out.size());
        return out;
    };
    b->h_yargs = bytes(ya);
    b->h_gargs = bytes(ga);
    b->h_cargs = bytes(ca);
    b->h_margs = bytes(ma);
    b->h_fdesc = bytes(fd);
    ml_status st;
    if ((st = upload(b, 0, &b->d_yargs, b->h_yargs, s)) != ML_OK) return st;
    if ((st = upload(b, 1, &b->d_gargs, b->h_gargs, s)) != ML_OK) return st;
    if ((st = upload(b, 2, &b->d_cargs, b->h_cargs, s)) != ML_OK) return st;
    if ((st = upload(b, 3, &b->d_margs, b->h_margs, s)) != ML_OK) return st;
    if ((st = upload(b, 4, &b->d_fdesc, b->h_fdesc, s)) != ML_OK) return st;
    if ((st = upload(b, 5, (void **)&b->d_maps, b->h_maps, s)) != ML_OK) return st;
    if ((st = upload(b, 6, (void **)&b->d_lev0, b->h_lev0, s)) != ML_OK) return st;
    if ((st = upload(b, 7, (void **)&b->d_ywork, b->h_ywork, s)) != ML_OK) return st;
    if ((st = upload(b, 8, (void **)&b->d_gwork, b->h_gwork, s)) != ML_OK) return st;
    if ((st = upload(b, 9, (void **)&b->d_mwork, b->h_mwork, s)) != ML_OK) return st;
    if ((st = upload(b, 10, (void **)&b->d_fwork, b->h_fwork, s)) != ML_OK) return st;
    return ML_OK;
}

// Enqueue steps s0 .. s0+count-1 of a sequence that starts at a fold boundary.
// Events around one launch while tracing (never inside a capture: traced steps run
// without the graph).
struct BatchScope {
    ml_batch *b;
    cudaStream_t s;
    int kind;
    cudaEvent_t a = nullptr;
    BatchScope(ml_batch *b_, cudaStream_t s_, int k) : b(b_), s(s_), kind(k) {
        if (b->timing) {
            cudaEventCreate(&a);
            cudaEventRecord(a, s);
        }
    }
    ~BatchScope() {
        if (a) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            cudaEventRecord(e, s);
            b->timed.push_back({a, e, kind});
        }
    }
};

template <typename T>
ml_status enqueue(ml_batch *b, int s0, int count, bool fold_tail, cudaStream_t s) {
    const int nyw = (int)b->h_ywork.size(), ngw = (int)b->h_gwork.size(), nmw = (int)b->h_mwork.size();
    const int nfw = (int)b->h_fwork.size();
    const int grid = b->blocks_per_sm > 0 ? std::min(nyw, b->blocks_per_sm * b->sms) : nyw;
    for (int q = 0; q < count; q++) {
        const int st = s0 + q;
        if (nmw > 0) {
            {
                BatchScope bs(b, s, 0);
                MolBatch<T> mb{(const MolArgs<T> *)b->d_margs, b->d_lev0, b->d_mwork, st, b->mol_two_level ? 1 : 0};
                CK(launch_molecules_batch<T>(mb, nmw, s));
            }
            {
                BatchScope bs(b, s, 4);
                CurBatch<T> cb{(const CurArgs<T> *)b->d_cargs, b->d_gwork};
                CK(launch_current_batch<T>(cb, ngw, s, b->pdl));
            }
            b->launches += 2;
        }
        {
            BatchScope bs(b, s, 1);
            YeeBatch<T> yb{(const YeeArgs<T> *)b->d_yargs, b->d_maps, b->d_lev0, b->d_ywork, nyw, b->d_boff, st,
                           st % DFT_KMAX, b->bodies};
            CK(launch_yee_batch<T>(yb, grid, s, b->pdl && nmw > 0));
            // periodic images of the level each periodic instance just wrote
            for (size_t i = 0; i < b->g.size(); i++) {
                const ml_grid *gi = b->g[i];
                if (!(gi->per[0] | gi->per[1] | gi->per[2])) continue;
                const int wrote = 1 - ((b->h_lev0[i] + st) & 1);
                CK(launch_images<T>(image_args<T>(gi, wrote), s));
                b->launches++;
            }
        }
        b->launches++;
        const bool period_end = st % DFT_KMAX == DFT_KMAX - 1;
        if (nfw > 0 && (period_end || (fold_tail && q == count - 1))) {
            BatchScope bs(b, s, 3);
            const int first = st - st % DFT_KMAX;
            FoldBatch<T> fbt{(const FoldDesc<T> *)b->d_fdesc, b->d_fwork, st - first + 1, b->d_boff, first,
                             b->g[0]->dt};
            CK(launch_fold_batch<T>(fbt, nfw, s));
            b->launches++;
        }
    }
    return ML_OK;
}

template <typename T>
ml_status batch_step(ml_batch *b, long long nsteps, cudaStream_t s) {
    // every grid starts with an empty DFT ring
    for (ml_grid *g : b->g) {
        ml_status st = fold_planes<T>(g, s);
        if (st != ML_OK) return st;
    }
    ml_status st = prepare<T>(b, s);
    if (st != ML_OK) return st;
    CK(cudaMemsetAsync(b->d_boff, 0, sizeof(long long), s));
    const int grid = b->blocks_per_sm > 0 ? b->blocks_per_sm : 0;
    std::vector<long long> sig = {(long long)b->h_ywork.size(), (long long)b->h_gwork.size(),
                                  (long long)b->h_mwork.size(), (long long)b->h_fwork.size(), grid,
                                  (long long)(uintptr_t)b->d_yargs, (long long)(uintptr_t)b->d_gargs,
                                  (long long)(uintptr_t)b->d_cargs, (long long)(uintptr_t)b->d_margs,
                                  (long long)(uintptr_t)b->d_fdesc, (long long)(uintptr_t)b->d_maps,
                                  (long long)(uintptr_t)b->d_lev0, (long long)(uintptr_t)b->d_ywork,
                                  (long long)(uintptr_t)b->d_gwork, (long long)(uintptr_t)b->d_mwork,
                                  (long long)(uintptr_t)b->d_fwork};
    // the periodic-image launches bake in the level each periodic instance writes
    long long nper = 0;
    for (size_t i = 0; i < b->g.size(); i++)
        if (b->g[i]->per[0] | b->g[i]->per[1] | b->g[i]->per[2]) {
            nper++;
            sig.push_back(((long long)i << 1) | (b->h_lev0[i] & 1));
        }
    const long long reps = (b->use_graph && !b->timing) ? nsteps / SEQ : 0;
    if (reps > 0) {
        if (b->exec && sig != b->sig) drop_graph(b);
        if (!b->exec) {
            CK(cudaStreamSynchronize(s));  // the argument arrays are in place before capture
            CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
            const long long l0 = b->launches;
            ml_status e = enqueue<T>(b, 0, SEQ, false, b->cap_stream);
            cudaError_t te = launch_tick(b->d_boff, SEQ, b->cap_stream);
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamEndCapture(b->cap_stream, &graph);
            b->launches = l0;
            if (e != ML_OK) {
                if (graph) cudaGraphDestroy(graph);
                return e;
            }
            if (te != cudaSuccess || ce != cudaSuccess)
                return fail(ML_ERR_CUDA, std::string("batch graph capture: ") +
                                             cudaGetErrorString(te != cudaSuccess ? te : ce));
            b->graph = graph;
            CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
            b->sig = sig;
        }
        const long long per = (long long)(b->h_mwork.size() ? 2 : 0) + 1 + nper;
        for (long long r = 0; r < reps; r++) {
            CK(cudaGraphLaunch(b->exec, s));
            b->launches += SEQ * per + (b->h_fwork.empty() ? 0 : SEQ / DFT_KMAX) + 1;
        }
    }
    const int rest = (int)(nsteps - reps * SEQ);
    if (rest > 0) {
        st = enqueue<T>(b, 0, rest, true, s);
        if (st != ML_OK) return st;
        CK(launch_tick(b->d_boff, rest, s));
        b->launches++;
    }
    for (ml_grid *g : b->g) {
        g->step += nsteps;
        if (nsteps & 1) g->cur ^= 1;
        g->nsamp = 0;
        g->samp_step0 = g->step;
    }
    return ML_OK;
}

}  // namespace

ml_status ml_batch_create(ml_grid *const *grids, int n, ml_batch **out) {
    if (!grids || n < 1 || !out) return fail(ML_ERR_INVALID_ARG, "batch needs at least one grid");
    for (int i = 0; i < n; i++) {
        if (!grids[i]) return fail(ML_ERR_INVALID_ARG, "null grid in batch");
        if (grids[i]->prec != grids[0]->prec) return fail(ML_ERR_INVALID_ARG, "batch grids differ in precision");
        if (grids[i]->dt != grids[0]->dt) return fail(ML_ERR_INVALID_ARG, "batch grids differ in time step");
        for (int j = 0; j < i; j++)
            if (grids[j] == grids[i]) return fail(ML_ERR_INVALID_ARG, "grid appears twice in batch");
    }
    ml_batch *b = new ml_batch();
    b->g.assign(grids, grids + n);
    b->prec = grids[0]->prec;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    b->blocks_per_sm = b->prec ? 1 : 3;
    if (const char *ev = std::getenv("ML_PDL")) b->pdl = std::atoi(ev) != 0;
    // the smallest body set of the field pass that covers every instance's tiles (a
    // vacuum grid's CPML tiles may take the table body: it reads the background entry)
    b->bodies = YEE_BODIES_VACUUM;
    for (ml_grid *g : b->g) {
        if (g->bodies == YEE_BODIES_ALL) b->bodies = YEE_BODIES_ALL;
        else if (g->bodies == YEE_BODIES_TABLES && b->bodies == YEE_BODIES_VACUUM) b->bodies = YEE_BODIES_TABLES;
    }
    {
        ml_status st = dev_alloc(b->mem, (void **)&b->d_boff, sizeof(long long));
        if (st != ML_OK) {
            ml_batch_destroy(b);
            return st;
        }
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        // kernel attributes are set outside any capture
        YeeBatch<double> yd{};
        YeeBatch<float> yf{};
        yd.bodies = yf.bodies = b->bodies;
        e = b->prec ? launch_yee_batch<double>(yd, 1, b->cap_stream) : launch_yee_batch<float>(yf, 1, b->cap_stream);
    }
    if (e != cudaSuccess) {
        ml_batch_destroy(b);
        return fail(ML_ERR_CUDA, std::string("batch create: ") + cudaGetErrorString(e));
    }
    *out = b;
    return ML_OK;
}

ml_status ml_batch_destroy(ml_batch *b) {
    if (!b) return ML_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    dev_free_all(b->mem);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
    return ML_OK;
}

ml_status ml_batch_step(ml_batch *b, int64_t nsteps, void *stream) {
    if (!b) return fail(ML_ERR_INVALID_ARG, "null batch");
    if (nsteps < 0) return fail(ML_ERR_INVALID_ARG, "negative step count");
    if (nsteps == 0) return ML_OK;
    cudaStream_t s = (cudaStream_t)stream;
    return b->prec ? batch_step<double>(b, nsteps, s) : batch_step<float>(b, nsteps, s);
}

ml_status ml_batch_set_tuning(ml_batch *b, int blocks_per_sm, int use_graph) {
    if (!b || blocks_per_sm < 0) return fail(ML_ERR_INVALID_ARG, "bad tuning");
    b->blocks_per_sm = blocks_per_sm;
    b->use_graph = use_graph != 0;
    return ML_OK;
}

int64_t ml_batch_launch_count(const ml_batch *b) { return b ? b->launches : -1; }

ml_status ml_batch_set_timing(ml_batch *b, int enable) {
    if (!b) return fail(ML_ERR_INVALID_ARG, "null batch");
    b->timing = enable != 0;
    return ML_OK;
}

ml_status ml_batch_timing(ml_batch *b, double *ms, int64_t *counts) {
    if (!b) return fail(ML_ERR_INVALID_ARG, "null batch");
    double t[6] = {0, 0, 0, 0, 0, 0};
    int64_t c[6] = {0, 0, 0, 0, 0, 0};
    for (auto &x : b->timed) {
        CK(cudaEventSynchronize(x.b));
        float f = 0.f;
        CK(cudaEventElapsedTime(&f, x.a, x.b));
        t[x.kind] += f;
        c[x.kind]++;
        cudaEventDestroy(x.a);
        cudaEventDestroy(x.b);
    }
    b->timed.clear();
    for (int q = 0; q < 6; q++) {
        if (ms) ms[q] = t[q];
        if (counts) counts[q] = c[q];
    }
    return ML_OK;
}

// Autotuner: time `trial_steps` batched steps for each field-pass grid shape (blocks
// per SM 1..occupancy, or one block per work item), restoring every grid's state after
// each trial, and keep the fastest.
ml_status ml_batch_autotune(ml_batch *b, int trial_steps, void *stream, int *blocks_per_sm, double *ms_out) {
    if (!b || trial_steps < 1) return fail(ML_ERR_INVALID_ARG, "bad autotune arguments");
    cudaStream_t s = (cudaStream_t)stream;
    // device snapshot of every grid (the trials advance them)
    std::vector<std::vector<Blob>> blobs;
    std::vector<void *> snaps;
    std::vector<long long> steps;
    std::vector<int> curs;
    DevList snap_mem;  // returned when the call ends
    for (ml_grid *g : b->g) {
        // empty DFT rings first, so that the snapshot plus the host counters is the state
        ml_status st = g->prec ? fold_planes<double>(g, s) : fold_planes<float>(g, s);
        if (st != ML_OK) return st;
        blobs.push_back(state_blobs(g));
        size_t n = 0;
        for (auto &x : blobs.back()) n += x.bytes;
        void *p = nullptr;
        st = dev_alloc(snap_mem.v, &p, n);
        if (st != ML_OK) return st;
        snaps.push_back(p);
        char *o = (char *)p;
        for (auto &x : blobs.back()) {
            CK(cudaMemcpyAsync(o, x.p, x.bytes, cudaMemcpyDeviceToDevice, s));
            o += x.bytes;
        }
        steps.push_back(g->step);
        curs.push_back(g->cur);
    }
    auto restore_all = [&]() -> ml_status {
        for (size_t i = 0; i < b->g.size(); i++) {
            const char *o = (const char *)snaps[i];
            for (auto &x : blobs[i]) {
                CK(cudaMemcpyAsync(x.p, o, x.bytes, cudaMemcpyDeviceToDevice, s));
                o += x.bytes;
            }
            b->g[i]->step = steps[i];
            b->g[i]->cur = curs[i];
            b->g[i]->nsamp = 0;
            b->g[i]->samp_step0 = steps[i];
        }
        return ML_OK;
    };
    const int occ = b->prec ? 1 : 3;
    std::vector<int> cand = {0};
    for (int q = 1; q <= occ; q++) cand.push_back(q);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int best_c = b->blocks_per_sm;
    const int keep = b->blocks_per_sm;
    for (int c : cand) {
        b->blocks_per_sm = c;
        ml_status st = ml_batch_step(b, trial_steps, s);  // warm-up (and graph capture)
        if (st == ML_OK) st = restore_all();
        if (st != ML_OK) {
            b->blocks_per_sm = keep;
            return st;
        }
        CK(cudaEventRecord(e0, s));
        st = ml_batch_step(b, trial_steps, s);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (st == ML_OK) st = restore_all();
        if (st != ML_OK) {
            b->blocks_per_sm = keep;
            return st;
        }
        if (ms < best) {
            best = ms;
            best_c = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaStreamSynchronize(s));
    b->blocks_per_sm = best_c;
    if (blocks_per_sm) *blocks_per_sm = best_c;
    if (ms_out) *ms_out = best;
    return ML_OK;
}
