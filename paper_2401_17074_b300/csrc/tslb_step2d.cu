// D2Q9 variant of the TSLB step (the same third-order recursive
// regularisation on the two-dimensional lattice D1Q3 x D1Q3).
//
// State: six moment fields per node in two vector arrays, V0 = (u_x, u_y,
// rho - 1, Pi_xy) at element 0 and V1 = (Pi_xx, Pi_yy) at element 4 * fs
// (FP32; 24 bytes per node and buffer, so one step moves 48 bytes per node).
//
// Step: every node x gathers the post-collision populations of its eight
// neighbours x - c_i (Eq. pushLB in pull form), each rebuilt from the
// neighbour's moments by third-order Hermite regularisation (Eq. eqts,
// Eq. noneqts, Luo forcing of Sec. 3.1), and sums the new moments (Sec. 2.1).
// As in three dimensions the map factorises into 1-D passes of the three
// 1-D populations p+ = a0 + a1 + 2 a2, p- = a0 - a1 + 2 a2, p0 = 4 (a0 - a2)
// (integer weights {1, 4, 1}, phi_2 = 3c^2 - 1; sums carry 36 x the
// deviation).  Each warp owns 32 columns (30 outputs and two halo lanes) and
// marches y: the y pass runs on the march window in registers, the x pass
// through warp shuffles.  Warps share nothing, so the kernel has no barriers
// and no shared-memory exchange; each thread stages its column's next rows
// through its own shared-memory slots (cp.async, a ring of four rows fetched
// three rows ahead).
//
// Faces: periodic x; periodic or halfway bounce-back y.  The wall layers
// contribute no deviation, and the populations that return from a wall -- the
// node's own populations leaving towards it, reversed -- are added in closed
// form from the y-contractions B_kx = A_kx0 - s A_kx1 + 2 A_kx2 of the node's
// post-collision modes (s = +1 at the lower wall, -1 at the upper).
#include <algorithm>

#include "tslb_internal.cuh"

namespace tslb {
namespace {

constexpr int XOUT2 = 30;   // output columns per warp (lanes 1..30)
constexpr int WARPS2 = 16;   // independent warps per CTA
constexpr int SLOTS2 = 4;   // prefetch ring (rows)
constexpr int AHEAD2 = 3;   // rows fetched ahead
constexpr int NT2 = 32 * WARPS2;
constexpr int ROWB = 32;    // staged bytes per thread and row: V0 (16) at +0, V1 (8) at +16, padded so
                            // every 16-byte copy lands 16-byte aligned

// 1/36 as a two-term constant (the second term rounded to FP32): quotients by
// 36 land within about half an ulp.
constexpr float INV36_HI = 0x1.c71c72p-6f;
constexpr float INV36_LO = -0x1.c71c72p-33f;
__device__ __forceinline__ float div36(float x) { return fmaf(x, INV36_HI, x * INV36_LO); }

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async2(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void commit2() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void wait_ahead2() { asm volatile("cp.async.wait_group %0;" ::"n"(AHEAD2) : "memory"); }

struct Pops1 {
    float pp, pm, c;
};
__device__ __forceinline__ Pops1 pops_3(float a0, float a1, float a2) {
    const float e = fmaf(2.0f, a2, a0);
    return {e + a1, e - a1, a0 - a2};
}

// y populations of the three kx groups of a source node (unscaled Hermite
// coefficients in, the mode scales of the scaled basis folded in):
//   kx = 0: (A00, A01, A02) = (rho - 1, 3 j_y, 1.5 h_yy)
//   kx = 1: (A10, A11, A12) = (3 j_x, 9 h_xy, 4.5 h_xyy)
//   kx = 2: (A20, A21)      = (1.5 h_xx, 4.5 h_xxy)
// with j = rho (u + F), h2 = rho u u + P, h3_aab = u_a (h2_ab + P_ab) + u_b P_aa,
// P = (1 - omega) Pi (non-equilibrium velocity = u on every stored node).
// Also the y-contractions B_kx of the node's modes towards the wall at s.
__device__ __forceinline__ void ypops2(float drho, float ux, float uy, float pxx, float pyy, float pxy, float Fx,
                                       float Fy, float om, Pops1 P[3], float s, float B[3]) {
    const float rho = 1.0f + drho;
    const float Pxx = om * pxx, Pyy = om * pyy, Pxy = om * pxy;
    const float rux = rho * ux, ruy = rho * uy;
    const float jx = fmaf(rho, Fx, rux), jy = fmaf(rho, Fy, ruy);
    const float hxx = fmaf(rux, ux, Pxx), hyy = fmaf(ruy, uy, Pyy);
    const float hxy = fmaf(rux, uy, Pxy);
    const float txy = hxy + Pxy;
    const float hxxy = fmaf(ux, txy, uy * Pxx), hxyy = fmaf(uy, txy, ux * Pyy);
    {
        const float e = fmaf(3.0f, hyy, drho);
        P[0] = {fmaf(3.0f, jy, e), fmaf(-3.0f, jy, e), fmaf(-1.5f, hyy, drho)};
    }
    {
        const float t = 3.0f * jx, e = fmaf(9.0f, hxyy, t);
        P[1] = {fmaf(9.0f, hxy, e), fmaf(-9.0f, hxy, e), fmaf(-4.5f, hxyy, t)};
    }
    {
        const float t = 1.5f * hxx;
        P[2] = {fmaf(4.5f, hxxy, t), fmaf(-4.5f, hxxy, t), t};
    }
    // B_kx = A_kx0 - s A_kx1 + 2 A_kx2
    B[0] = fmaf(3.0f, hyy, fmaf(-3.0f * s, jy, drho));
    B[1] = fmaf(9.0f, hxyy, fmaf(-9.0f * s, hxy, 3.0f * jx));
    B[2] = fmaf(-4.5f * s, hxxy, 1.5f * hxx);
}

__global__ void __launch_bounds__(NT2) step2d_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                     Geometry g, Physics p, int ychunk, int ntx) {
    __shared__ __align__(16) char ring[SLOTS2][NT2 * ROWB];
    const int lane = threadIdx.x & 31;
    const int wid = blockIdx.x * WARPS2 + (threadIdx.x >> 5);
    const int tx = wid % ntx, ty = wid / ntx;
    const int y0 = ty * ychunk;
    if (y0 >= g.ny) return;  // whole warp: the kernel has no barriers
    const int y1 = min(y0 + ychunk, g.ny);
    const int np = y1 - y0 + 2;  // march rows y0-1 .. y1
    const int x = tx * XOUT2 + lane - 1;
    const unsigned xl = (unsigned)((x + g.nx) % g.nx);
    const bool store = lane >= 1 && lane <= XOUT2 && x < g.nx;
    const bool yper = g.bc[2] == TSLB_BC_PERIODIC;
    const long long fs = g.fstride;
    char* slot0 = &ring[0][threadIdx.x * ROWB];

    // stored row of march row ys, or -1 for a wall layer (zero deviation)
    auto row_of = [&](int ys) -> int {
        if (yper) return (ys + g.ny) % g.ny;
        return (ys < 0 || ys >= g.ny) ? -1 : ys;
    };
    auto fetch = [&](int j) {
        const int yl = row_of(y0 - 1 + j);
        const unsigned n = xl + (unsigned)g.nx * (unsigned)(yl < 0 ? 0 : yl);
        char* b = slot0 + (j & (SLOTS2 - 1)) * (NT2 * ROWB);
        if (j < np && yl >= 0 && TSLB_IN_RANGE(n, g.plane, p.err)) {
            cp_async2<16>(smem_addr(b), src + (size_t)n * 4);
            cp_async2<8>(smem_addr(b + 16), src + 4 * fs + (size_t)n * 2);
        }
        commit2();
    };
    // Launched with programmatic stream serialisation: global memory only
    // after the preceding step's grid has completed (see the factored kernel).
    asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
    for (int q = 0; q < AHEAD2; ++q) fetch(q);

    const float om = p.omega1, Fx = p.F[0], Fy = p.F[1];
    // y window: p+ of rows ys-2 and ys-1, c of row ys-1
    float pp2[3] = {0.f, 0.f, 0.f}, pp1[3] = {0.f, 0.f, 0.f}, c1[3] = {0.f, 0.f, 0.f};
    float Blo[3] = {0.f, 0.f, 0.f}, Bhi[3] = {0.f, 0.f, 0.f};
    for (int j = 0; j < np; ++j) {
        fetch(j + AHEAD2);
        wait_ahead2();
        const int ys = y0 - 1 + j;
        const int yl = row_of(ys);
        Pops1 P[3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        if (yl >= 0) {
            const char* b = slot0 + (j & (SLOTS2 - 1)) * (NT2 * ROWB);
            const float4 a = *reinterpret_cast<const float4*>(b);
            const float2 c2 = *reinterpret_cast<const float2*>(b + 16);
            const bool lo_wall = !yper && ys == 0, hi_wall = !yper && ys == g.ny - 1;
            float B[3];
            ypops2(a.z, a.x, a.y, c2.x, c2.y, a.w, Fx, Fy, om, P, lo_wall ? 1.0f : -1.0f, B);
            if (lo_wall) {
                Blo[0] = B[0]; Blo[1] = B[1]; Blo[2] = B[2];
            }
            if (hi_wall) {
                Bhi[0] = B[0]; Bhi[1] = B[1]; Bhi[2] = B[2];
            }
        }
        if (j >= 2) {
            // ---- y moments of output row ys - 1 -------------------------------
            float Z[3][3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float L = pp2[k], R = P[k].pm;
                Z[k][2] = L + R;
                Z[k][1] = L - R;
                Z[k][0] = fmaf(4.0f, c1[k], Z[k][2]);
            }
            // ---- x pass: groups r over kx --------------------------------------
            float M[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const Pops1 X = pops_3(Z[0][r], Z[1][r], Z[2][r]);
                const float Lx = __shfl_up_sync(0xffffffffu, X.pp, 1);
                const float Rx = __shfl_down_sync(0xffffffffu, X.pm, 1);
                const float sLR = Lx + Rx;
                M[r][0] = fmaf(4.0f, X.c, sLR);
                M[r][1] = Lx - Rx;
                M[r][2] = sLR;
            }
            float D0 = M[0][0], Jx = M[0][1], Jy = M[1][0];
            float Sxx = M[0][2], Syy = M[2][0], Sxy = M[1][1];
            const int yo = ys - 1;
            if (!yper && (yo == 0 || yo == g.ny - 1)) {
                // populations returning from the wall(s) next to this row
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 0 ? yo != 0 : yo != g.ny - 1) continue;
                    const float s = side == 0 ? 1.0f : -1.0f;
                    const float* B = side == 0 ? Blo : Bhi;
                    const float b6 = 6.0f * B[0];
                    D0 += b6;
                    Jx = fmaf(-2.0f, B[1], Jx);
                    Jy = fmaf(s, b6, Jy);
                    Sxx = fmaf(2.0f, B[0], fmaf(4.0f, B[2], Sxx));
                    Syy += b6;
                    Sxy = fmaf(-2.0f * s, B[1], Sxy);
                }
            }
            // ---- new moments: rho - 1 = D0/36, u = J/(36 + D0),
            //      Pi_ab = (S_ab - J_a u_b - delta_ab D0/3) / 36
            const float inv = rcp_refined(36.0f + D0);
            const float ux = Jx * inv, uy = Jy * inv, d3 = D0 * (1.0f / 3.0f);
            if (store && TSLB_IN_RANGE(xl + (long long)g.nx * yo, g.plane, p.err)) {
                const unsigned n = xl + (unsigned)g.nx * (unsigned)yo;
                reinterpret_cast<float4*>(dst)[n] =
                    make_float4(ux, uy, div36(D0), div36(Sxy - Jx * uy));
                reinterpret_cast<float2*>(dst + 4 * fs)[n] =
                    make_float2(div36(Sxx - fmaf(Jx, ux, d3)), div36(Syy - fmaf(Jy, uy, d3)));
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            pp2[k] = pp1[k];
            pp1[k] = P[k].pp;
            c1[k] = P[k].c;
        }
    }
}

// ---- codecs and diagnostics of the 2-D state ----------------------------------

__global__ void encode2d_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                                const double* __restrict__ pi, float* __restrict__ dst, Geometry g, long long fnx,
                                long long fN) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane) return;
    const long long xi = n % g.nx, yi = n / g.nx;
    const long long node = (xi + g.lo[0]) + fnx * (yi + g.lo[1]);
    const float pxx = pi ? (float)pi[node] : 0.f, pyy = pi ? (float)pi[fN + node] : 0.f;
    const float pxy = pi ? (float)pi[3 * fN + node] : 0.f;
    reinterpret_cast<float4*>(dst)[n] =
        make_float4((float)u[node], (float)u[fN + node], (float)(rho[node] - 1.0), pxy);
    reinterpret_cast<float2*>(dst + 4 * g.fstride)[n] = make_float2(pxx, pyy);
}

__global__ void decode2d_kernel(const float* __restrict__ src, double* __restrict__ rho, double* __restrict__ u,
                                double* __restrict__ pi, Geometry g, long long fnx, long long fny) {
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long fN = fnx * fny;
    if (node >= fN) return;
    const long long xi = node % fnx - g.lo[0], yi = node / fnx - g.lo[1];
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 c = make_float2(0.f, 0.f);
    if (xi >= 0 && xi < g.nx && yi >= 0 && yi < g.ny) {
        const long long n = xi + g.nx * yi;
        a = reinterpret_cast<const float4*>(src)[n];
        c = reinterpret_cast<const float2*>(src + 4 * g.fstride)[n];
    }
    if (rho) rho[node] = 1.0 + (double)a.z;
    if (u) {
        u[node] = a.x;
        u[fN + node] = a.y;
        u[2 * fN + node] = 0.0;
    }
    if (pi) {
        pi[node] = c.x;
        pi[fN + node] = c.y;
        pi[2 * fN + node] = 0.0;
        pi[3 * fN + node] = a.w;
        pi[4 * fN + node] = 0.0;
        pi[5 * fN + node] = 0.0;
    }
}

// [mass, jx, jy, jz, ke, shear_sum, max_speed, nonfinite], as the 3-D diagnostics.
__global__ void __launch_bounds__(256) diag2d_partial_kernel(const float* __restrict__ src, Geometry g,
                                                             double shear_scale, double* __restrict__ part) {
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const bool ywalls = g.bc[2] == TSLB_BC_BOUNCEBACK;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < g.plane;
         n += (long long)gridDim.x * blockDim.x) {
        const float4 a = reinterpret_cast<const float4*>(src)[n];
        if (!(isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w))) {
            acc[7] += 1.0;
            continue;
        }
        const double r = 1.0 + (double)a.z, ux = a.x, uy = a.y;
        acc[0] += r;
        acc[1] += r * ux;
        acc[2] += r * uy;
        const double u2 = ux * ux + uy * uy;
        acc[4] += 0.5 * r * u2;
        acc[6] = fmax(acc[6], sqrt(u2));
        if (ywalls) {
            const long long yi = n / g.nx;
            if (yi == 0) acc[5] -= shear_scale * (double)a.w;
            if (yi == g.ny - 1) acc[5] += shear_scale * (double)a.w;
        }
    }
    __shared__ double red[8][8];
    const int ln = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 8; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_xor_sync(0xffffffffu, v, o);
            v = (k == 6) ? fmax(v, t) : v + t;
        }
        if (ln == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int k = threadIdx.x;
        double v = red[k][0];
        for (int i = 1; i < 8; ++i) v = (k == 6) ? fmax(v, red[k][i]) : v + red[k][i];
        part[blockIdx.x * 8 + k] = v;
    }
}

__global__ void diag2d_final_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 8) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v = (k == 6) ? fmax(v, part[b * 8 + k]) : v + part[b * 8 + k];
    out[k] = v;
}

}  // namespace

cudaError_t launch_step2d(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    const Geometry& g = h->g;
    const int ntx = (g.nx + XOUT2 - 1) / XOUT2;
    // As many independent warps as fit on the GPU at once (one wave: a second,
    // partial wave would cost a whole chunk's time), in y chunks that are long
    // against their two halo rows.
    static int resident[64] = {};
    const int dev = h->device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!resident[dev]) {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step2d_kernel, NT2, 0);
        if (e != cudaSuccess) return e;
        resident[dev] = per_sm > 0 ? per_sm : 1;
    }
    const int sms = h->sm_count > 0 ? h->sm_count : 148;
    const long long want = (long long)sms * resident[dev] * WARPS2;
    int nchunk = (int)std::min<long long>(g.ny, std::max<long long>(1, want / ntx));
    const int ychunk = (g.ny + nchunk - 1) / nchunk;
    nchunk = (g.ny + ychunk - 1) / ychunk;
    const long long warps = (long long)ntx * nchunk;
    const unsigned blocks = (unsigned)((warps + WARPS2 - 1) / WARPS2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(NT2);
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, step2d_kernel, (const float*)src, (float*)dst, g, p, ychunk, ntx);
}

cudaError_t launch_encode2d(const tslb_s* h, const double* rho, const double* u, const double* pi, void* dst) {
    const long long total = h->g.plane;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    encode2d_kernel<<<blocks, 256, 0, h->stream>>>(rho, u, pi, (float*)dst, h->g, h->dims[0],
                                                   h->dims[0] * h->dims[1]);
    return cudaGetLastError();
}

cudaError_t launch_decode2d(const tslb_s* h, const void* src, double* rho, double* u, double* pi) {
    const long long fN = h->dims[0] * h->dims[1];
    const unsigned blocks = (unsigned)((fN + 255) / 256);
    decode2d_kernel<<<blocks, 256, 0, h->stream>>>((const float*)src, rho, u, pi, h->g, h->dims[0], h->dims[1]);
    return cudaGetLastError();
}

cudaError_t launch_diag2d(const tslb_s* h, const void* src, double* out_dev) {
    diag2d_partial_kernel<<<h->diag_blocks, 256, 0, h->stream>>>((const float*)src, h->g, 1.0 - 0.5 * h->omega,
                                                                 h->diag_part);
    diag2d_final_kernel<<<1, 32, 0, h->stream>>>(h->diag_part, h->diag_blocks, out_dev);
    return cudaGetLastError();
}

}  // namespace tslb
