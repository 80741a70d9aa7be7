// ml_gather_static: regularised molecular fields from a caller-owned field, for
// callers that cannot allocate device memory.
//
// Some applications cannot let a library call cudaMalloc: their device memory is
// reserved up front by their own allocator (a framework's caching pool, a fixed
// budget on a shared GPU), or the call sits on a latency-critical path where an
// allocation, which may synchronise the device, is not acceptable.  This entry
// point needs no grid handle and allocates nothing: its only scratch is the
// file-scope device array below, of a fixed maximum size, held by every GPU that
// loads the library until the process exits.
//
// Two kernels: one block per molecule, whose first warp computes the molecule's six
// normalised 1D weight vectors once into shared memory, and whose sixteen warps (one
// per plane of the kernel window) write the planes' weighted field sums into the
// scratch array (every slot the second kernel reads is written by the first, so
// nothing needs clearing); one warp per molecule then adds the planes in a fixed
// order and applies the coupling.
// Calls share the scratch: calls that overlap on the GPU (for example on two
// streams) race, so issue them one after another.
#include <cmath>
#include <mutex>
#include <string>

#include "maxlink.h"
#include "ml_internal.cuh"

namespace {

constexpr int SG_PLANES = ml::WMAX;  // window planes per molecule (2 ceil(3 sigma) + 2 <= 16)

static __device__ __align__(256) float g_sg_scratch[ML_STATIC_GATHER_MAX_MOLECULES * SG_PLANES * 3];

struct SgArgs {
    const float *E;   // 3 x (nz, ny, nx)
    int nx, ny, nz, px, py, pz;  // dims and periodic flags
    int nmol;
    const double *pos, *sigma, *gamma;
    float *scratch;   // device address of g_sg_scratch
    float *out;
};

// The six normalised 1D weight vectors of molecule m ([axis][stagger][t], zero past the
// window), computed by one warp into `w`: sample t of axis ax at (s + t) + stag/2, centre
// p.  The exponent is taken relative to the nearest sample, so the largest weight is
// exactly 1 and a narrow kernel cannot underflow to 0/0 (the normalisation removes the
// common factor).  Three exps per lane.
__device__ __forceinline__ void sg_weights(const double (&p)[3], const int (&s)[3], int W, double sg, float (&w)[6][16]) {
    const int lane = threadIdx.x & 31;
    const double inv = 1.0 / (2.0 * sg * sg);
    double e[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int v = lane + 32 * k;  // vector v / 16 = 2 ax + stag, entry t = v % 16
        const int ax = (v >> 4) >> 1, stag = (v >> 4) & 1, t = v & 15;
        // nearest sample of this vector: distance of the centre to the sample grid
        const double f = p[ax] - 0.5 * stag;
        const double dn = f - floor(f + 0.5);
        const double d = (double)(s[ax] + t) + 0.5 * stag - p[ax];
        e[k] = t < W ? exp(-(d * d - dn * dn) * inv) : 0.0;
    }
    // sums of each 16-entry vector: lanes 0-15 and 16-31 hold one vector per k
#pragma unroll
    for (int k = 0; k < 3; k++) {
        double sum = e[k];
        for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const int v = lane + 32 * k;
        w[v >> 4][v & 15] = (float)(e[k] / sum);
    }
    __syncwarp();
}

__device__ __forceinline__ int sg_wrap(int c, int n, int per, bool &ok) {
    if (c >= 0 && c < n) return c;
    if (!per) { ok = false; return 0; }
    return ((c % n) + n) % n;
}

// Molecules whose width or position the entry point cannot take get NaN outputs.
__device__ __forceinline__ bool sg_valid(const SgArgs &a, int m) {
    const double sg = a.sigma[m];
    bool ok = sg > 0.0 && ceil(3.0 * sg) <= 7.0;
    for (int ax = 0; ax < 3; ax++) ok = ok && fabs(a.pos[3 * m + ax]) < 1.0e9;
    return ok;
}

// grid: molecules, SG_PLANES warps per block: warp dz takes plane dz of the window.
// Lane = (dx in 0..15, row parity).
__global__ void __launch_bounds__(SG_PLANES * 32) sg_partial_kernel(const SgArgs a) {
    __shared__ float w[6][16];
    const int m = blockIdx.x, dz = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (m >= a.nmol) return;
    const bool valid = sg_valid(a, m);  // uniform over the block
    int R = 0, W = 0, s[3] = {0, 0, 0};
    if (valid) {
        const double sg = a.sigma[m];
        R = (int)ceil(3.0 * sg);
        W = 2 * R + 2;
        double p[3];
        for (int ax = 0; ax < 3; ax++) {
            p[ax] = a.pos[3 * m + ax];
            s[ax] = (int)floor(p[ax]) - R;
        }
        if (dz == 0) sg_weights(p, s, W, sg, w);
    }
    __syncthreads();
    float part[3] = {0.f, 0.f, 0.f};
    if (valid) {
        const int dx = lane & 15, ly = lane >> 4;
        bool okz = dz < W;
        const int z = sg_wrap(s[2] + dz, a.nz, a.pz, okz);
        bool okx = dx < W;
        const int x = sg_wrap(s[0] + dx, a.nx, a.px, okx);
        if (okz && okx) {
            // component c is sampled half a cell along c (Yee staggering): w[2 ax + stag]
            const float wx0 = w[0][dx], wx1 = w[1][dx], wz0 = w[4][dz], wz1 = w[5][dz];
            const long long N = (long long)a.nx * a.ny * a.nz;
            for (int dy = ly; dy < W; dy += 2) {
                bool oky = true;
                const int y = sg_wrap(s[1] + dy, a.ny, a.py, oky);
                if (!oky) continue;
                const float wy0 = w[2][dy], wy1 = w[3][dy];
                const long long f = ((long long)z * a.ny + y) * a.nx + x;
                part[0] += a.E[f] * (wx1 * wy0 * wz0);
                part[1] += a.E[N + f] * (wx0 * wy1 * wz0);
                part[2] += a.E[2 * N + f] * (wx0 * wy0 * wz1);
            }
        }
    }
    for (int c = 0; c < 3; c++) {
        float v = part[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) a.scratch[((long long)m * SG_PLANES + dz) * 3 + c] = v;
    }
}

// one warp per molecule: the SG_PLANES plane sums added by a fixed xor tree
__global__ void sg_reduce_kernel(const SgArgs a) {
    const int m = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (m >= a.nmol) return;
    const bool ok = sg_valid(a, m);
    for (int c = 0; c < 3; c++) {
        float v = lane < SG_PLANES ? a.scratch[((long long)m * SG_PLANES + lane) * 3 + c] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) a.out[3 * m + c] = ok ? (float)a.gamma[m] * v : __int_as_float(0x7fc00000);
    }
}

std::mutex g_mu;
float *g_ptr[256] = {};  // device address of g_sg_scratch, per device ordinal

ml_status sg_fail(ml_status s, const std::string &msg) {
    ml::set_last_error(msg);
    return s;
}

}  // namespace

ml_status ml_gather_static(const float *E, int nx, int ny, int nz, const int *periodic, int nmol, const double *pos,
                           const double *sigma, const double *gamma, float *out, void *stream) {
    if (nmol < 0 || nmol > ML_STATIC_GATHER_MAX_MOLECULES)
        return sg_fail(ML_ERR_INVALID_ARG, "nmol must be 0.." + std::to_string(ML_STATIC_GATHER_MAX_MOLECULES) +
                                               " (the fixed scratch holds that many molecules)");
    if (nx < 1 || ny < 1 || nz < 1 || !periodic) return sg_fail(ML_ERR_INVALID_ARG, "bad grid dimensions");
    if (nmol == 0) return ML_OK;
    if (!E || !pos || !sigma || !gamma || !out) return sg_fail(ML_ERR_INVALID_ARG, "null pointer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) return sg_fail(ML_ERR_CUDA, "cudaGetDevice failed");
    if (stream) {
        // the scratch address is the current device's: the stream must belong to it
        int sdev = -1;
        e = cudaStreamGetDevice((cudaStream_t)stream, &sdev);
        if (e != cudaSuccess || sdev != dev)
            return sg_fail(ML_ERR_INVALID_ARG, "the stream does not belong to the current device");
    }
    float *scratch = nullptr;
    {
        // set-up on the first call for this device (the device is current here)
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_sg_scratch);
            if (e != cudaSuccess || !p)
                return sg_fail(ML_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_ptr[dev] = static_cast<float *>(p);
        }
        scratch = g_ptr[dev];
    }
    SgArgs a;
    a.E = E;
    a.nx = nx; a.ny = ny; a.nz = nz;
    a.px = periodic[0] ? 1 : 0; a.py = periodic[1] ? 1 : 0; a.pz = periodic[2] ? 1 : 0;
    a.nmol = nmol;
    a.pos = pos; a.sigma = sigma; a.gamma = gamma;
    a.scratch = scratch;
    a.out = out;
    cudaStream_t s = (cudaStream_t)stream;
    sg_partial_kernel<<<nmol, SG_PLANES * 32, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return sg_fail(ML_ERR_CUDA, std::string("partial kernel: ") + cudaGetErrorString(e));
    sg_reduce_kernel<<<(nmol + 3) / 4, 128, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return sg_fail(ML_ERR_CUDA, std::string("reduce kernel: ") + cudaGetErrorString(e));
    return ML_OK;
}
