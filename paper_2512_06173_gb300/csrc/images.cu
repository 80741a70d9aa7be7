// Periodic ghost images of the six field arrays of one time level, written after each
// field pass of a grid with a periodic axis (the field pass stores its own cells only).
#include <type_traits>

#include "ml_internal.cuh"

namespace ml {

// Periodic images after a field pass: one thread per ghost cell on the faces of the
// periodic axes (a cell on two faces is written twice, with the same value).  The cell
// takes the value of its image inside the grid, found by wrapping each coordinate; a
// ghost that lies outside along a wall axis stays 0.  Reading only interior cells makes
// the order of the writes irrelevant.
template <typename T>
__global__ void image_kernel(const ImgArgs<T> a) {
    const long long X = a.nx + 2, Y = a.ny + 2, Z = a.nz + 2;
    const long long fx = a.per[0] ? 2 * Y * Z : 0, fy = a.per[1] ? 2 * X * Z : 0, fz = a.per[2] ? 2 * X * Y : 0;
    const long long n = fx + fy + fz;
    // x faces with nx a multiple of 8: a thread copies the whole 32-byte sector that holds
    // its row's ghost (x = -8..-1 from nx-8..nx-1, or x = nx..nx+7 from 0..7), so every
    // access is a full aligned sector; the extra cells are padding that nothing reads, and
    // they get their periodic images too
    const bool xsec = a.per[0] && (a.nx % 8) == 0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        int i, j, k;
        if (t < fx) {
            const long long r = t % (Y * Z);
            j = (int)(r % Y) - 1;
            k = (int)(r / Y) - 1;
            i = t >= Y * Z ? a.nx : -1;
            if (xsec) {
                const bool oy = j < 0 || j >= a.ny, oz = k < 0 || k >= a.nz;
                if ((oy && !a.per[1]) || (oz && !a.per[2])) continue;
                const int sj = j < 0 ? j + a.ny : (j >= a.ny ? j - a.ny : j);
                const int sk = k < 0 ? k + a.nz : (k >= a.nz ? k - a.nz : k);
                const long long drow = (long long)(k + 1) * a.plane + (long long)(j + 1) * a.px;
                const long long srow = (long long)(sk + 1) * a.plane + (long long)(sj + 1) * a.px;
                const long long dst = drow + (i < 0 ? XO - 8 : a.nx + XO);
                const long long src = srow + (i < 0 ? a.nx + XO - 8 : XO);
                // (rows start 128-byte aligned and nx % 8 == 0: both ends are 16-byte aligned)
                using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
                constexpr int NV = 8 * (int)sizeof(T) / 16;
#pragma unroll
                for (int c = 0; c < 6; c++) {
                    const V *sp = reinterpret_cast<const V *>(a.f[c] + src);
                    V *dp = reinterpret_cast<V *>(a.f[c] + dst);
                    V v[NV];
#pragma unroll
                    for (int q = 0; q < NV; q++) v[q] = sp[q];
#pragma unroll
                    for (int q = 0; q < NV; q++) dp[q] = v[q];
                }
                continue;
            }
        } else if (t < fx + fy) {
            const long long u = t - fx, r = u % (X * Z);
            i = (int)(r % X) - 1;
            k = (int)(r / X) - 1;
            j = u >= X * Z ? a.ny : -1;
        } else {
            const long long u = t - fx - fy, r = u % (X * Y);
            i = (int)(r % X) - 1;
            j = (int)(r / X) - 1;
            k = u >= X * Y ? a.nz : -1;
        }
        const bool ox = i < 0 || i >= a.nx, oy = j < 0 || j >= a.ny, oz = k < 0 || k >= a.nz;
        if ((ox && !a.per[0]) || (oy && !a.per[1]) || (oz && !a.per[2])) continue;
        const int si = i < 0 ? i + a.nx : (i >= a.nx ? i - a.nx : i);
        const int sj = j < 0 ? j + a.ny : (j >= a.ny ? j - a.ny : j);
        const int sk = k < 0 ? k + a.nz : (k >= a.nz ? k - a.nz : k);
        const long long dst = (long long)(k + 1) * a.plane + (long long)(j + 1) * a.px + (i + XO);
        const long long src = (long long)(sk + 1) * a.plane + (long long)(sj + 1) * a.px + (si + XO);
        T v[6];
#pragma unroll
        for (int c = 0; c < 6; c++) v[c] = a.f[c][src];
#pragma unroll
        for (int c = 0; c < 6; c++) a.f[c][dst] = v[c];
    }
}

template <typename T>
cudaError_t launch_images(const ImgArgs<T> &a, cudaStream_t s) {
    const long long X = a.nx + 2, Y = a.ny + 2, Z = a.nz + 2;
    const long long n = (a.per[0] ? 2 * Y * Z : 0) + (a.per[1] ? 2 * X * Z : 0) + (a.per[2] ? 2 * X * Y : 0);
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    image_kernel<T><<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_images<float>(const ImgArgs<float> &, cudaStream_t);
template cudaError_t launch_images<double>(const ImgArgs<double> &, cudaStream_t);

}  // namespace ml
