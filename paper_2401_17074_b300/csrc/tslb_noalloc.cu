// Diagnostics reduction that allocates nothing (tslb_diagnostics_noalloc).
//
// Same FP64 sums as tslb_diagnostics, but over moment arrays the caller
// owns (the full-lattice FP64 layout that tslb_get_moments writes) and with
// the per-block partial sums kept in a fixed file-scope device array instead
// of memory obtained from cudaMalloc.  For callers that cannot allocate
// device memory where they want the numbers: a fixed device-memory budget
// that is already spent, a framework allocator that owns every byte of the
// device, or a latency-bound loop in which cudaMalloc / cudaFree (which may
// synchronise the device) are not acceptable.
#include <cstring>
#include <mutex>
#include <string>

#include "tslb_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_NODES_PER_THREAD = 64;
constexpr long long NA_NODES_PER_BLOCK = (long long)NA_THREADS * NA_NODES_PER_THREAD;  // 16384
constexpr int NA_MAX_BLOCKS = 4096;
constexpr int NA_SUMS = 8;
static_assert(NA_NODES_PER_BLOCK * NA_MAX_BLOCKS == TSLB_NOALLOC_MAX_NODES, "limit mismatch");

// Partial sums of up to NA_MAX_BLOCKS blocks (256 KB).  Every device that
// loads this library holds one copy until the process exits.  Each call
// overwrites the slots of the blocks it launches before reading them, so no
// slot has to start at zero; two calls that overlap on the GPU race here.
static __device__ __align__(256) double g_noalloc_partials[NA_MAX_BLOCKS * NA_SUMS];

// Host-side device address of g_noalloc_partials, looked up once per device
// (on the first call with that device current) and kept for the life of the
// process.  It belongs to the device's primary context: after cudaDeviceReset
// on that device the cached address is stale and this entry point must not be
// called again in the process.
std::mutex g_mu;
double* g_partials_addr[64] = {};

int na_fail(int code, const std::string& m) {
    tslb::set_global_error(m);
    return code;
}

// Sums over interior nodes: [mass, jx, jy, jz, ke, shear_sum, max_speed, nonfinite].
__global__ void __launch_bounds__(NA_THREADS) noalloc_partial_kernel(const double* __restrict__ rho,
                                                                   const double* __restrict__ u,
                                                                   const double* __restrict__ pi, long long fnx,
                                                                   long long fny, long long fN, int lo0, int lo1,
                                                                   int lo2, long long nx, long long ny,
                                                                   long long total, int ywalls, double shear_scale,
                                                                   double* __restrict__ partials) {
    double acc[NA_SUMS] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long first = (long long)blockIdx.x * NA_NODES_PER_BLOCK;
    const long long last = min(first + NA_NODES_PER_BLOCK, total);
    for (long long n = first + threadIdx.x; n < last; n += NA_THREADS) {
        const long long xi = n % nx, yi = (n / nx) % ny, zi = n / (nx * ny);
        const long long node = (xi + lo0) + fnx * ((yi + lo1) + fny * (zi + lo2));
        const double r = rho[node], ux = u[node], uy = u[fN + node], uz = u[2 * fN + node];
        // a node counts as non-finite if any of its ten moments is NaN or Inf,
        // as in tslb_diagnostics
        bool finite = isfinite(r) && isfinite(ux) && isfinite(uy) && isfinite(uz);
        double pxy = 0.0;
        if (pi) {
#pragma unroll
            for (int k = 0; k < 6; ++k) finite = finite && isfinite(pi[k * fN + node]);
            pxy = pi[3 * fN + node];
        }
        if (!finite) {
            acc[7] += 1.0;
            continue;
        }
        acc[0] += r;
        acc[1] += r * ux;
        acc[2] += r * uy;
        acc[3] += r * uz;
        const double u2 = ux * ux + uy * uy + uz * uz;
        acc[4] += 0.5 * r * u2;
        acc[6] = fmax(acc[6], sqrt(u2));
        if (ywalls) {
            if (yi == 0) acc[5] -= shear_scale * pxy;
            if (yi == ny - 1) acc[5] += shear_scale * pxy;
        }
    }
    __shared__ double red[NA_SUMS][NA_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < NA_SUMS; ++k) {
        double x = acc[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (k == 6) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < NA_SUMS) {
        const int k = threadIdx.x;
        double x = red[k][0];
        for (int w = 1; w < NA_THREADS / 32; ++w) x = (k == 6) ? fmax(x, red[k][w]) : x + red[k][w];
        partials[(long long)blockIdx.x * NA_SUMS + k] = x;
    }
}

__global__ void noalloc_final_kernel(const double* __restrict__ partials, int nblocks, double shear_norm,
                                     double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= NA_SUMS) return;
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) x = (k == 6) ? fmax(x, partials[b * NA_SUMS + k]) : x + partials[b * NA_SUMS + k];
    out[k] = (k == 5) ? x * shear_norm : x;
}

}  // namespace

extern "C" int tslb_diagnostics_noalloc(const double* rho, const double* u, const double* pi, const int64_t dims[3],
                                        const int bc[6], double tau, void* stream, double* out) {
    tslb::set_global_error("");
    if (!rho || !u || !dims || !bc || !out) return na_fail(TSLB_ERR_INVALID, "null argument");
    if (!(tau > 0.5)) return na_fail(TSLB_ERR_INVALID, "tau must be > 1/2");
    long long ext[3];
    int lo[3];
    for (int a = 0; a < 3; ++a) {
        if (bc[2 * a] < TSLB_BC_PERIODIC || bc[2 * a] > TSLB_BC_NEE_WALL || bc[2 * a + 1] < TSLB_BC_PERIODIC ||
            bc[2 * a + 1] > TSLB_BC_NEE_WALL)
            return na_fail(TSLB_ERR_INVALID, "unknown boundary code");
        const bool per = bc[2 * a] == TSLB_BC_PERIODIC;
        if (per != (bc[2 * a + 1] == TSLB_BC_PERIODIC))
            return na_fail(TSLB_ERR_INVALID, "an axis mixes periodic and non-periodic faces");
        if (dims[a] < (per ? 1 : 3)) return na_fail(TSLB_ERR_INVALID, "axis too short");
        if (dims[a] > ((int64_t)1 << 30)) return na_fail(TSLB_ERR_INVALID, "axis too long");
        lo[a] = per ? 0 : 1;
        ext[a] = per ? dims[a] : dims[a] - 2;
    }
    // the interior count, checked factor by factor so the product cannot overflow
    const long long lim = TSLB_NOALLOC_MAX_NODES;
    if (ext[0] > lim || ext[1] > lim / ext[0] || ext[2] > lim / (ext[0] * ext[1]))
        return na_fail(TSLB_ERR_INVALID, "more interior nodes than TSLB_NOALLOC_MAX_NODES (2^26); use tslb_diagnostics");
    const long long total = ext[0] * ext[1] * ext[2];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(TSLB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return na_fail(TSLB_ERR_UNSUPPORTED, "device ordinal above 63");
    double* partials = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_partials_addr[dev]) {
            // The array's name is only a host-side stand-in; the kernels need its
            // device address on this device.
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_partials);
            if (e != cudaSuccess)
                return na_fail(TSLB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_partials_addr[dev] = static_cast<double*>(p);
        }
        partials = g_partials_addr[dev];
    }
    const int nblocks = (int)((total + NA_NODES_PER_BLOCK - 1) / NA_NODES_PER_BLOCK);
    const bool ywalls = bc[2] == TSLB_BC_BOUNCEBACK || bc[2] == TSLB_BC_NEE_WALL;
    const double shear_scale = 1.0 - 0.5 / tau;
    const double shear_norm = ywalls ? 1.0 / (2.0 * (double)ext[0] * (double)ext[2]) : 0.0;
    const long long fN = (long long)dims[0] * dims[1] * dims[2];
    cudaStream_t s = (cudaStream_t)stream;
    if (nblocks > 0)
        noalloc_partial_kernel<<<nblocks, NA_THREADS, 0, s>>>(rho, u, pi, dims[0], dims[1], fN, lo[0], lo[1], lo[2],
                                                              ext[0], ext[1], total, ywalls ? 1 : 0, shear_scale,
                                                              partials);
    noalloc_final_kernel<<<1, 32, 0, s>>>(partials, nblocks, shear_norm, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(TSLB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return TSLB_OK;
}
