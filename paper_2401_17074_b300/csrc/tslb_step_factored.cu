// Sum-factorised TSLB step: one CTA marches a 30 x 16 column tile along z.
//
// Physics: every node x gathers the post-collision populations of its
// neighbours x - c_i (Eq. pushLB in pull form), each rebuilt from the
// neighbour's moments by third-order Hermite regularisation (Eq. eqts,
// Eq. noneqts, Luo forcing of Sec. 3.1), and sums the new moments (Sec. 2.1).
//
// Because D3Q27 is the tensor product D1Q3 x D1Q3 x D1Q3 with product
// weights and product Hermite polynomials, the map "17 mode coefficients of
// the neighbours -> 10 moments of the gathered populations" factorises into
// three 1-D passes.  Each pass turns up to three mode coefficients
// (a0, a1, a2) of a source node into its three 1-D populations
//     p+ = a0 + a1 + 2 a2,  p- = a0 - a1 + 2 a2,  p0 = 4 (a0 - a2)
// (integer weights {1, 4, 1}, phi_2 = 3c^2 - 1), shifts p+ by +1 and p- by -1
// along the axis, and takes the 1-D moments at the destination
//     M0 = p+(x-1) + p0(x) + p-(x+1),  M1 = p+(x-1) - p-(x+1),  M2 = p+(x-1) + p-(x+1).
// Order of the passes: z in registers (each thread owns an (x, y) column and
// marches z, so z-neighbours are the previous / next loop iterations), then y
// through shared memory (warps are rows), then x through warp shuffles
// (lanes are columns).  Halo: lanes 0 and 31 and the first and last warp
// recompute the border columns / rows of the tile.
//
// Faces: periodic axes wrap the loads; a free-slip face mirrors the 1-D pass
// (the population entering from the wall side is the node's own population
// leaving towards it, Sec. 2.3 walls as specular reflection); a bounce-back y
// face zeroes the entering deviation and adds the reversed populations of the
// node itself (halfway bounce-back); inflow / outflow z faces enter the march
// as ghost planes (Eq. neq_final for the inflow, the adjacent layer's moments
// for the outflow, Sec. 3.2).
#include "tslb_internal.cuh"

#include <algorithm>

namespace tslb {
namespace {

constexpr int XOUT = 30;             // output columns per warp (lanes 1..30)
constexpr int WROWS = 18;            // warps per CTA; rows 1..16 are outputs
constexpr int YOUT = WROWS - 2;
constexpr int NT = 32 * WROWS;
constexpr int YSLOTS = 18;           // y-exchange values per thread: 9 groups x {p+, p-}
constexpr size_t SMEM_BYTES = sizeof(float) * 2 * YSLOTS * NT;

struct Pops {
    float pp, pm, c;
};
__device__ __forceinline__ Pops pops3(float a0, float a1, float a2) {
    const float e = fmaf(2.0f, a2, a0);
    return {e + a1, e - a1, 4.0f * (a0 - a2)};
}
__device__ __forceinline__ Pops pops2(float a0, float a1) { return {a0 + a1, a0 - a1, 4.0f * a0}; }
__device__ __forceinline__ Pops pops1(float a0) { return {a0, a0, 4.0f * a0}; }

// Moments of one node; `off` is the node's 32-bit offset inside a field.
template <class Codec>
__device__ __forceinline__ void load_moments(const typename Codec::T* __restrict__ src, long long fstride,
                                             unsigned off, const Physics& p, float m[NFIELDS]) {
#pragma unroll
    for (int f = 0; f < NFIELDS; ++f) m[f] = Codec::dec(src[f * fstride + off], field_scale(f, p));
}

// Interior plane stored at march position zs (periodic wrap, inflow / outflow ghosts).
__device__ __forceinline__ int plane_of(int zs, const Geometry& g, bool zper, bool& inflow_ghost) {
    inflow_ghost = false;
    if (zs < 0) {
        if (zper) return zs + g.nz;
        inflow_ghost = true;
        return 0;
    }
    if (zs >= g.nz) return zper ? zs - g.nz : g.nz - 1;  // outflow ghost copies the last layer
    return zs;
}

template <class Codec, bool XFREE>
__global__ void __launch_bounds__(NT, 1)
    step_factored_kernel(const typename Codec::T* __restrict__ src, typename Codec::T* __restrict__ dst, Geometry g,
                         Physics p, int zchunk) {
    extern __shared__ float ysm[];  // [2][YSLOTS][NT]
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int x = blockIdx.x * XOUT + lane - 1;
    const int y = blockIdx.y * YOUT + warp - 1;
    const bool yper = g.bc[2] == TSLB_BC_PERIODIC;
    const bool ybb = g.bc[2] == TSLB_BC_BOUNCEBACK;
    const bool yfs = g.bc[2] == TSLB_BC_FREESLIP;
    const bool zper = g.bc[4] == TSLB_BC_PERIODIC;

    // Column this thread loads (always inside the stored box).
    const int xl = XFREE ? min(max(x, 0), g.nx - 1) : (x + g.nx) % g.nx;
    const int yl = yper ? (y + g.ny) % g.ny : min(max(y, 0), g.ny - 1);
    const unsigned col = (unsigned)xl + (unsigned)g.nx * (unsigned)yl;
    const unsigned plane = (unsigned)g.plane;
    const bool store = lane >= 1 && lane <= XOUT && x < g.nx && warp >= 1 && warp <= YOUT && y < g.ny;
    const bool xlo_mirror = XFREE && x == 0, xhi_mirror = XFREE && x == g.nx - 1;
    // warp-uniform row roles in the y pass
    const bool row_lo = y == 0, row_hi = y == g.ny - 1;
    const int below = warp > 0 ? tid - 32 : tid;
    const int above = warp < WROWS - 1 ? tid + 32 : tid;

    const int z0 = blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, g.nz);

    float zL2[8], zL1[8], zC[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) zL2[k] = zL1[k] = zC[k] = 0.0f;
    int buf = 0;

    // one plane of moments in flight ahead of the plane being processed
    float mn[NFIELDS];
    {
        bool ig;
        const int zl = plane_of(z0 - 1, g, zper, ig);
        load_moments<Codec>(src, g.fstride, col + plane * (unsigned)zl, p, mn);
    }
    for (int zs = z0 - 1; zs <= z1; ++zs) {
        // ---- source plane zs: moments -> 17 modes -> z populations --------
        bool inflow_ghost;
        const int zl = plane_of(zs, g, zper, inflow_ghost);
        const unsigned idx = col + plane * (unsigned)zl;
        float m[NFIELDS];
#pragma unroll
        for (int f = 0; f < NFIELDS; ++f) m[f] = mn[f];
        if (zs < z1) {
            bool ig;
            const int zn = plane_of(zs + 1, g, zper, ig);
            load_moments<Codec>(src, g.fstride, col + plane * (unsigned)zn, p, mn);
        }
        float A[NMODES];
        if (inflow_ghost) {
            const float uBz = inflow_uz(p, (long long)xl + g.lo[0], (long long)yl + g.lo[1]);
            post_modes(m[F_DRHO], 0.f, 0.f, uBz, m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], 0.f, 0.f, 0.f, p.omega1, A);
        } else {
            float F0 = p.F[0], F1 = p.F[1], F2 = p.F[2];
            if (p.force) {
                F0 = __ldg(p.force + idx);
                F1 = __ldg(p.force + g.fstride + idx);
                F2 = __ldg(p.force + 2 * g.fstride + idx);
            }
            post_modes(m[F_DRHO], m[F_UX], m[F_UY], m[F_UZ], m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], F0, F1, F2,
                       p.omega1, A);
        }
        Pops P[8];
        P[0] = pops3(A[M000], A[M001], A[M002]);  // (k1,k2) = (0,0)
        P[1] = pops3(A[M100], A[M101], A[M102]);  // (1,0)
        P[2] = pops3(A[M010], A[M011], A[M012]);  // (0,1)
        P[3] = pops2(A[M200], A[M201]);           // (2,0)
        P[4] = pops2(A[M020], A[M021]);           // (0,2)
        P[5] = pops2(A[M110], A[M111]);           // (1,1)
        P[6] = pops1(A[M210]);                    // (2,1)
        P[7] = pops1(A[M120]);                    // (1,2)

        if (zs >= z0 + 1) {
            // ---- z moments of plane z = zs - 1 ------------------------------
            float Z[8][3];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float L = zL2[k], R = P[k].pm;
                Z[k][2] = L + R;
                Z[k][1] = L - R;
                Z[k][0] = Z[k][2] + zC[k];
            }
            // ---- y pass: groups (k1, r) over k2 -----------------------------
            Pops Q[9];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                Q[0 + r] = pops3(Z[0][r], Z[2][r], Z[4][r]);  // k1 = 0: k2 = 0, 1, 2
                Q[3 + r] = pops3(Z[1][r], Z[5][r], Z[7][r]);  // k1 = 1
                Q[6 + r] = pops2(Z[3][r], Z[6][r]);           // k1 = 2
            }
            float* sb = ysm + buf * (YSLOTS * NT);
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                sb[(2 * j) * NT + tid] = Q[j].pp;
                sb[(2 * j + 1) * NT + tid] = Q[j].pm;
            }
            __syncthreads();
            // Y[k1][q][r] for (q, r) in {(0,0),(1,0),(2,0),(0,1),(1,1),(0,2)}
            float Y[3][6];
#pragma unroll
            for (int k1 = 0; k1 < 3; ++k1) {
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int j = 3 * k1 + r;
                    float L = sb[(2 * j) * NT + below];
                    float R = sb[(2 * j + 1) * NT + above];
                    if (row_lo) {
                        if (ybb) L = 0.0f;
                        else if (yfs) L = sb[(2 * j + 1) * NT + tid];
                    }
                    if (row_hi) {
                        if (ybb) R = 0.0f;
                        else if (yfs) R = sb[(2 * j) * NT + tid];
                    }
                    const float s = L + R;
                    if (r == 0) {
                        Y[k1][0] = s + Q[j].c;  // q = 0
                        Y[k1][1] = L - R;       // q = 1
                        Y[k1][2] = s;           // q = 2
                    } else if (r == 1) {
                        Y[k1][3] = s + Q[j].c;  // (q, r) = (0, 1)
                        Y[k1][4] = L - R;       // (1, 1)
                    } else {
                        Y[k1][5] = s + Q[j].c;  // (0, 2)
                    }
                }
            }
            buf ^= 1;
            // ---- x pass: groups (q, r) over k1 ------------------------------
            float Mo[6][3];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const Pops X = pops3(Y[0][k], Y[1][k], Y[2][k]);
                float L = __shfl_up_sync(0xffffffffu, X.pp, 1);
                float R = __shfl_down_sync(0xffffffffu, X.pm, 1);
                if (xlo_mirror) L = X.pm;
                if (xhi_mirror) R = X.pp;
                const float s = L + R;
                Mo[k][0] = s + X.c;
                Mo[k][1] = L - R;
                Mo[k][2] = s;
            }
            float D0 = Mo[0][0];
            float J[3] = {Mo[0][1], Mo[1][0], Mo[3][0]};
            float S[6] = {Mo[0][2], Mo[2][0], Mo[5][0], Mo[1][1], Mo[3][1], Mo[4][0]};
            const int z = zs - 1;
            const unsigned oidx = col + plane * (unsigned)z;
            // ---- halfway bounce-back on the wall-adjacent rows --------------
            if (ybb && (row_lo || row_hi)) {
                float mo[NFIELDS];
                load_moments<Codec>(src, g.fstride, oidx, p, mo);
                float F0 = p.F[0], F1 = p.F[1], F2 = p.F[2];
                if (p.force) {
                    F0 = __ldg(p.force + oidx);
                    F1 = __ldg(p.force + g.fstride + oidx);
                    F2 = __ldg(p.force + 2 * g.fstride + oidx);
                }
                float Ao[NMODES];
                post_modes(mo[F_DRHO], mo[F_UX], mo[F_UY], mo[F_UZ], mo[F_UX], mo[F_UY], mo[F_UZ], &mo[F_PXX], F0,
                           F1, F2, p.omega1, Ao);
                const int cy = row_lo ? 1 : -1;  // direction arriving from the wall
#pragma unroll
                for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
                    for (int cx = -1; cx <= 1; ++cx) {
                        const float gi = pop_dev216(Ao, -cx, -cy, -cz);
                        D0 += gi;
                        J[0] = fmaf(gi, (float)cx, J[0]);
                        J[1] = fmaf(gi, (float)cy, J[1]);
                        J[2] = fmaf(gi, (float)cz, J[2]);
                        S[0] = fmaf(gi, (float)(cx * cx), S[0]);
                        S[1] += gi;
                        S[2] = fmaf(gi, (float)(cz * cz), S[2]);
                        S[3] = fmaf(gi, (float)(cx * cy), S[3]);
                        S[4] = fmaf(gi, (float)(cx * cz), S[4]);
                        S[5] = fmaf(gi, (float)(cy * cz), S[5]);
                    }
            }
            float out[NFIELDS];
            finish_moments(D0, J, S, out);
            if (store) {
#pragma unroll
                for (int f = 0; f < NFIELDS; ++f) dst[f * g.fstride + oidx] = Codec::enc(out[f], field_inv_scale(f, p));
            }
        }
        // ---- advance the z window ------------------------------------------
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            zL2[k] = zL1[k];
            zL1[k] = P[k].pp;
            zC[k] = P[k].c;
        }
    }
}

template <class Codec, bool XFREE>
cudaError_t launch_t(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    auto kern = step_factored_kernel<Codec, XFREE>;
    static bool configured[64] = {};
    int dev = h->device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const tslb::Geometry& g = h->g;
    const unsigned bx = (unsigned)((g.nx + XOUT - 1) / XOUT);
    const unsigned by = (unsigned)((g.ny + YOUT - 1) / YOUT);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // z chunks: fill whole waves of one CTA per SM while keeping chunks long
    // (each chunk re-reads two extra planes).
    const long long tiles = (long long)bx * by;
    int best_n = 1;
    double best = 0.0;
    for (int n = 1; n <= 16 && n <= g.nz; ++n) {
        const int len = (g.nz + n - 1) / n;
        const long long ctas = tiles * n;
        const long long waves = (ctas + sms - 1) / sms;
        const double eff = (double)ctas / (double)(waves * sms) * (double)len / (double)(len + 2);
        if (eff > best + 1e-3) {
            best = eff;
            best_n = n;
        }
    }
    const int zchunk = (g.nz + best_n - 1) / best_n;
    const unsigned bz = (unsigned)((g.nz + zchunk - 1) / zchunk);
    kern<<<dim3(bx, by, bz), NT, SMEM_BYTES, h->stream>>>((const typename Codec::T*)src, (typename Codec::T*)dst, g, p,
                                                         zchunk);
    return cudaGetLastError();
}

template <class Codec>
cudaError_t launch_codec(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    if (h->g.bc[0] == TSLB_BC_FREESLIP) return launch_t<Codec, true>(h, src, dst, p);
    return launch_t<Codec, false>(h, src, dst, p);
}

}  // namespace

bool factored_supports(const tslb_s* h) {
    (void)h;
    return true;
}

cudaError_t launch_step_factored(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    switch (h->precision) {
        case TSLB_FP32: return launch_codec<CodecF32>(h, src, dst, p);
        case TSLB_BF16: return launch_codec<CodecBF16>(h, src, dst, p);
        default: return launch_codec<CodecF16>(h, src, dst, p);
    }
}

}  // namespace tslb
