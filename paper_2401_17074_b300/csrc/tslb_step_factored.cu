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
// Memory path (default): each thread loads the 10 moments of its column with
// coalesced per-thread global loads, one plane ahead of the plane it is
// processing (register prefetch); stores go straight to global memory.
// Optional TMA feed (TSLB_KERNEL_FACTORED_TMA, when the row pitch is a multiple
// of 16 bytes): the plane tiles (+ halo) come into a three-stage shared-memory
// ring by cp.async.bulk.tensor, one box per field issued by the lanes of the
// last warp, completion counted on an mbarrier per stage; periodic wrap-around
// columns / rows come from small extra boxes in side regions that share the
// field stride, so only a thread's base offset depends on where its column
// lives.  On the B300 the register-prefetch feed measured faster (36.3 vs 29.1
// GLUPS on the 512 x 130 x 256 channel): the 217 KB ring leaves little L1 for
// the halo re-reads and every warp waits for a whole plane.
//
// Faces: periodic axes wrap; a free-slip face mirrors the 1-D pass (the
// population entering from the wall side is the node's own population leaving
// towards it: specular reflection); a bounce-back y face zeroes the entering
// deviation and adds the reversed populations of the node itself (halfway
// bounce-back); inflow / outflow z faces enter the march as ghost planes
// (Eq. neq_final for the inflow, the adjacent layer's moments for the
// outflow, Sec. 3.2).
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "tslb_internal.cuh"

namespace tslb {
namespace {

constexpr int XOUT = 30;   // output columns per warp (lanes 1..30)
constexpr int WROWS = 18;  // warps per CTA; rows 1..16 are outputs
constexpr int YOUT = WROWS - 2;
constexpr int NT = 32 * WROWS;
constexpr int YSLOTS = 18;  // y-exchange values per thread: 9 groups x {p+, p-}
constexpr int NSTAGE = 3;   // TMA ring depth (planes)
constexpr size_t YBYTES = sizeof(float) * 2 * YSLOTS * NT;

constexpr int align128(int b) { return (b + 127) / 128 * 128; }

// Shared-memory layout of one field of one stage, for element size E.
template <int E>
struct StageLayout {
    static constexpr int BX = E == 4 ? 36 : 40;  // main box width (covers 32 columns + alignment shift)
    static constexpr int XW = 16 / E;            // width of a wrap box (16 bytes)
    static constexpr int MAIN = 0;
    static constexpr int XL = MAIN + align128(WROWS * BX * E);
    static constexpr int XR = XL + align128(WROWS * XW * E);
    static constexpr int YB = XR + align128(WROWS * XW * E);
    static constexpr int YT = YB + align128(BX * E);
    static constexpr int CLB = YT + align128(BX * E);
    static constexpr int CRB = CLB + 128;
    static constexpr int CLT = CRB + 128;
    static constexpr int CRT = CLT + 128;
    static constexpr int FIELD = CRT + 128;  // bytes per field
    static constexpr int STAGE = NFIELDS * FIELD;
    static constexpr size_t SMEM = 128 + YBYTES + (size_t)NSTAGE * STAGE;
};

struct Pops {
    float pp, pm, c;
};
__device__ __forceinline__ Pops pops3(float a0, float a1, float a2) {
    const float e = fmaf(2.0f, a2, a0);
    return {e + a1, e - a1, 4.0f * (a0 - a2)};
}
__device__ __forceinline__ Pops pops2(float a0, float a1) { return {a0 + a1, a0 - a1, 4.0f * a0}; }
__device__ __forceinline__ Pops pops1(float a0) { return {a0, a0, 4.0f * a0}; }

// ---- PTX helpers: mbarrier + TMA ------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after about two seconds of SM clock.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 4000000000LL) return false;
    return true;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Tensor maps of one moment buffer: [field][z][y][x] viewed as a 4-D tensor
// (x, y, z, field); boxes main {BX, 18}, column wrap {XW, 18}, row wrap
// {BX, 1}, corner {XW, 1}, all one plane and one field deep.
struct TmaMaps {
    CUtensorMap main, col, row, corner;
};

// Moments of one node from global memory; `off` is the node's offset inside a field.
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

// Per-thread constants of the march.
struct Ctx {
    int tid, lane, warp, x, y, xl, yl;
    unsigned col, plane;
    int z0, z1, np;  // march covers planes z0-1 .. z1 (np of them)
    bool zper, ybb, store, row_lo, row_hi, zero_row, xlo_mirror, xhi_mirror;
    int offL, offR;      // y-exchange read offsets (relative to a slot base)
    uint32_t roff;       // byte offset of this thread's value inside a stage field (TMA path)
    uint32_t tx_bytes;   // bytes expected per stage fill (TMA path)
    bool xl_wrap, xr_wrap, yb_wrap, yt_wrap;
    int xa;              // first column of the main TMA box
    int issued;          // planes whose TMA fill has been issued (thread 0)
};

template <class Codec, bool XFREE, bool TMA>
struct Kernel {
    typedef typename Codec::T T;
    typedef StageLayout<(int)sizeof(T)> SL;

    // Issue the TMA boxes of march plane j into its stage.  Called by the
    // whole last warp: lane f issues the boxes of field f, so the ten fields go
    // out in one warp instruction instead of a serial loop on one thread.
    static __device__ __forceinline__ void fill(const Ctx& c, const Geometry& g, const TmaMaps& tm, char* stages,
                                                uint32_t bars, int j) {
        const int zs = c.z0 - 1 + j;
        bool ig;
        const int zl = plane_of(zs, g, c.zper, ig);
        const int s = j % NSTAGE;
        const uint32_t bar = bars + 8u * s;
        const uint32_t base = smem_u32(stages + (size_t)s * SL::STAGE);
        if (c.lane == 0) mbar_expect_tx(bar, c.tx_bytes);
        __syncwarp();
        const int y0m = (int)blockIdx.y * YOUT - 1;
        const int f = c.lane;
        if (f < NFIELDS) {
            const uint32_t fb = base + f * SL::FIELD;
            tma_load_4d(fb + SL::MAIN, &tm.main, bar, c.xa, y0m, zl, f);
            if (c.xl_wrap) tma_load_4d(fb + SL::XL, &tm.col, bar, g.nx - SL::XW, y0m, zl, f);
            if (c.xr_wrap) tma_load_4d(fb + SL::XR, &tm.col, bar, 0, y0m, zl, f);
            if (c.yb_wrap) tma_load_4d(fb + SL::YB, &tm.row, bar, c.xa, g.ny - 1, zl, f);
            if (c.yt_wrap) tma_load_4d(fb + SL::YT, &tm.row, bar, c.xa, 0, zl, f);
            if (c.xl_wrap && c.yb_wrap) tma_load_4d(fb + SL::CLB, &tm.corner, bar, g.nx - SL::XW, g.ny - 1, zl, f);
            if (c.xr_wrap && c.yb_wrap) tma_load_4d(fb + SL::CRB, &tm.corner, bar, 0, g.ny - 1, zl, f);
            if (c.xl_wrap && c.yt_wrap) tma_load_4d(fb + SL::CLT, &tm.corner, bar, g.nx - SL::XW, 0, zl, f);
            if (c.xr_wrap && c.yt_wrap) tma_load_4d(fb + SL::CRT, &tm.corner, bar, 0, 0, zl, f);
        }
    }

    // One march position j (plane zs = z0 - 1 + j).  ppOld holds p+ of plane
    // zs-2 on entry and p+ of plane zs on exit; cOld holds p0 of zs-1; cNew
    // receives p0 of zs.
    // Returns true (uniformly across the CTA) when a bounded wait gave up.
    static __device__ __forceinline__ bool plane_step(Ctx& c, const Geometry& g, const Physics& p,
                                                      const T* __restrict__ src, T* __restrict__ dst,
                                                      const TmaMaps& tm, char* stages, uint32_t bars, float* ysm,
                                                      float (&mn)[NFIELDS], int j, float (&ppOld)[8],
                                                      const float (&cOld)[8], float (&cNew)[8]) {
        int timed_out = 0;
        const int zs = c.z0 - 1 + j;
        bool inflow_ghost;
        const int zl = plane_of(zs, g, c.zper, inflow_ghost);
        const unsigned idx = c.col + c.plane * (unsigned)zl;
        float m[NFIELDS];
        if constexpr (TMA) {
            const int s = j % NSTAGE;
            if (!mbar_wait(bars + 8u * s, (uint32_t)((j / NSTAGE) & 1))) {
                timed_out = 1;
                if (p.err) atomicExch(p.err, 1);
            }
            const T* rp = reinterpret_cast<const T*>(stages + (size_t)s * SL::STAGE + c.roff);
#pragma unroll
            for (int f = 0; f < NFIELDS; ++f) m[f] = Codec::dec(rp[f * (SL::FIELD / (int)sizeof(T))], field_scale(f, p));
        } else {
#pragma unroll
            for (int f = 0; f < NFIELDS; ++f) m[f] = mn[f];
            if (zs < c.z1) {
                bool ig;
                const int zn = plane_of(zs + 1, g, c.zper, ig);
                load_moments<Codec>(src, g.fstride, c.col + c.plane * (unsigned)zn, p, mn);
            }
        }
        // ---- source plane: moments -> 17 modes -> z populations --------------
        float A[NMODES];
        if (inflow_ghost) {
            const float uBz = inflow_uz(p, (long long)c.xl + g.lo[0], (long long)c.yl + g.lo[1]);
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

        if (zs >= c.z0 + 1) {
            // ---- z moments of plane z = zs - 1 ------------------------------
            float Z[8][3];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float L = ppOld[k], R = P[k].pm;
                Z[k][2] = L + R;
                Z[k][1] = L - R;
                Z[k][0] = Z[k][2] + cOld[k];
            }
            // ---- y pass: groups (k1, r) over k2 -----------------------------
            Pops Q[9];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                Q[0 + r] = pops3(Z[0][r], Z[2][r], Z[4][r]);  // k1 = 0: k2 = 0, 1, 2
                Q[3 + r] = pops3(Z[1][r], Z[5][r], Z[7][r]);  // k1 = 1
                Q[6 + r] = pops2(Z[3][r], Z[6][r]);           // k1 = 2
            }
            float* sb = ysm + (j & 1) * (YSLOTS * NT);
            if (c.zero_row) {
                // ghost row beyond a bounce-back wall: the entering deviation is zero
#pragma unroll
                for (int q = 0; q < 2 * 9; ++q) sb[q * NT + c.tid] = 0.0f;
            } else {
#pragma unroll
                for (int jj = 0; jj < 9; ++jj) {
                    sb[(2 * jj) * NT + c.tid] = Q[jj].pp;
                    sb[(2 * jj + 1) * NT + c.tid] = Q[jj].pm;
                }
            }
            timed_out = __syncthreads_or(timed_out);
            // Y[k1][q][r] for (q, r) in {(0,0),(1,0),(2,0),(0,1),(1,1),(0,2)}
            float Y[3][6];
#pragma unroll
            for (int k1 = 0; k1 < 3; ++k1) {
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int jj = 3 * k1 + r;
                    const float L = sb[(2 * jj) * NT + c.offL];
                    const float R = sb[(2 * jj + 1) * NT + c.offR];
                    const float sLR = L + R;
                    if (r == 0) {
                        Y[k1][0] = sLR + Q[jj].c;  // q = 0
                        Y[k1][1] = L - R;          // q = 1
                        Y[k1][2] = sLR;            // q = 2
                    } else if (r == 1) {
                        Y[k1][3] = sLR + Q[jj].c;  // (q, r) = (0, 1)
                        Y[k1][4] = L - R;          // (1, 1)
                    } else {
                        Y[k1][5] = sLR + Q[jj].c;  // (0, 2)
                    }
                }
            }
            // ---- x pass: groups (q, r) over k1 ------------------------------
            float Mo[6][3];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const Pops X = pops3(Y[0][k], Y[1][k], Y[2][k]);
                float L = __shfl_up_sync(0xffffffffu, X.pp, 1);
                float R = __shfl_down_sync(0xffffffffu, X.pm, 1);
                if (XFREE) {
                    if (c.xlo_mirror) L = X.pm;
                    if (c.xhi_mirror) R = X.pp;
                }
                const float sLR = L + R;
                Mo[k][0] = sLR + X.c;
                Mo[k][1] = L - R;
                Mo[k][2] = sLR;
            }
            float D0 = Mo[0][0];
            float J[3] = {Mo[0][1], Mo[1][0], Mo[3][0]};
            float S[6] = {Mo[0][2], Mo[2][0], Mo[5][0], Mo[1][1], Mo[3][1], Mo[4][0]};
            const int z = zs - 1;
            const unsigned oidx = c.col + c.plane * (unsigned)z;
            // ---- halfway bounce-back on the wall-adjacent rows --------------
            if (c.ybb && (c.row_lo || c.row_hi)) {
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
                const int cy = c.row_lo ? 1 : -1;  // direction arriving from the wall
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
            if (c.store) {
#pragma unroll
                for (int f = 0; f < NFIELDS; ++f) dst[f * g.fstride + oidx] = Codec::enc(out[f], field_inv_scale(f, p));
            }
        } else {
            timed_out = __syncthreads_or(timed_out);
        }
        // every thread has read plane zs: its stage can take plane zs + NSTAGE
        if constexpr (TMA) {
            if (!timed_out && c.warp == WROWS - 1 && j + NSTAGE < c.np) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fill(c, g, tm, stages, bars, j + NSTAGE);
                c.issued = j + NSTAGE + 1;
            }
        }
        // ---- advance the z window --------------------------------------------
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            ppOld[k] = P[k].pp;
            cNew[k] = P[k].c;
        }
        return timed_out != 0;
    }
};

template <class Codec, bool XFREE, bool TMA>
__global__ void __launch_bounds__(NT, 1)
    step_factored_kernel(const typename Codec::T* __restrict__ src, typename Codec::T* __restrict__ dst, Geometry g,
                         Physics p, int zchunk, const __grid_constant__ TmaMaps tm) {
    typedef Kernel<Codec, XFREE, TMA> K;
    typedef typename K::SL SL;
    extern __shared__ __align__(128) char smem[];
    uint64_t* barp = reinterpret_cast<uint64_t*>(smem);         // [NSTAGE] mbarriers (128-byte header)
    float* ysm = reinterpret_cast<float*>(smem + 128);          // [2][YSLOTS][NT]
    char* stages = smem + 128 + YBYTES;                         // [NSTAGE][NFIELDS][FIELD]
    const uint32_t bars = smem_u32(barp);

    Ctx c;
    c.tid = threadIdx.x;
    c.lane = c.tid & 31;
    c.warp = c.tid >> 5;
    const int x0 = (int)blockIdx.x * XOUT, y0 = (int)blockIdx.y * YOUT;
    c.x = x0 + c.lane - 1;
    c.y = y0 + c.warp - 1;
    const bool xper = !XFREE;
    const bool yper = g.bc[2] == TSLB_BC_PERIODIC;
    c.ybb = g.bc[2] == TSLB_BC_BOUNCEBACK;
    const bool yfs = g.bc[2] == TSLB_BC_FREESLIP;
    c.zper = g.bc[4] == TSLB_BC_PERIODIC;
    c.xl = XFREE ? min(max(c.x, 0), g.nx - 1) : (c.x + g.nx) % g.nx;
    c.yl = yper ? (c.y + g.ny) % g.ny : min(max(c.y, 0), g.ny - 1);
    c.col = (unsigned)c.xl + (unsigned)g.nx * (unsigned)c.yl;
    c.plane = (unsigned)g.plane;
    c.store = c.lane >= 1 && c.lane <= XOUT && c.x < g.nx && c.warp >= 1 && c.warp <= YOUT && c.y < g.ny;
    c.xlo_mirror = XFREE && c.x == 0;
    c.xhi_mirror = XFREE && c.x == g.nx - 1;
    c.row_lo = c.y == 0;
    c.row_hi = c.y == g.ny - 1;
    c.zero_row = c.ybb && (c.y == -1 || c.y == g.ny);
    // y-exchange read offsets: the row below / above, or the node's own value
    // of the opposite population on a free-slip wall row
    c.offL = (yfs && c.row_lo) ? NT + c.tid : (c.warp > 0 ? c.tid - 32 : c.tid);
    c.offR = (yfs && c.row_hi) ? c.tid - NT : (c.warp < WROWS - 1 ? c.tid + 32 : c.tid);
    c.z0 = (int)blockIdx.z * zchunk;
    c.z1 = min(c.z0 + zchunk, g.nz);
    c.np = c.z1 - c.z0 + 2;

    float mn[NFIELDS];
    if constexpr (TMA) {
        constexpr int E = (int)sizeof(typename Codec::T);
        c.xa = (x0 - 1) & ~(SL::XW - 1);
        c.xl_wrap = xper && x0 == 0;
        c.xr_wrap = xper && x0 - 1 <= g.nx && g.nx <= x0 + XOUT;
        c.yb_wrap = yper && y0 == 0;
        c.yt_wrap = yper && y0 - 1 <= g.ny && g.ny <= y0 + YOUT;
        uint32_t per_field = WROWS * SL::BX;
        if (c.xl_wrap) per_field += WROWS * SL::XW;
        if (c.xr_wrap) per_field += WROWS * SL::XW;
        if (c.yb_wrap) per_field += SL::BX;
        if (c.yt_wrap) per_field += SL::BX;
        if (c.xl_wrap && c.yb_wrap) per_field += SL::XW;
        if (c.xr_wrap && c.yb_wrap) per_field += SL::XW;
        if (c.xl_wrap && c.yt_wrap) per_field += SL::XW;
        if (c.xr_wrap && c.yt_wrap) per_field += SL::XW;
        c.tx_bytes = per_field * NFIELDS * E;
        // where this thread's column lives inside a stage field
        const bool wl = xper && c.x == -1, wr = xper && c.x == g.nx;
        const bool wb = yper && c.y == -1, wt = yper && c.y == g.ny;
        const int row = c.warp, cx = c.x - c.xa;
        int off;
        if (wl && wb) off = SL::CLB + (SL::XW - 1) * E;
        else if (wr && wb) off = SL::CRB;
        else if (wl && wt) off = SL::CLT + (SL::XW - 1) * E;
        else if (wr && wt) off = SL::CRT;
        else if (wl) off = SL::XL + (row * SL::XW + SL::XW - 1) * E;
        else if (wr) off = SL::XR + (row * SL::XW) * E;
        else if (wb) off = SL::YB + cx * E;
        else if (wt) off = SL::YT + cx * E;
        else off = SL::MAIN + (row * SL::BX + cx) * E;
        c.roff = (uint32_t)off;
        if (c.tid == 0) {
            for (int s = 0; s < NSTAGE; ++s) mbar_init(bars + 8u * s, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        c.issued = 0;
        if (c.warp == WROWS - 1)
            for (int j = 0; j < NSTAGE && j < c.np; ++j) {
                K::fill(c, g, tm, stages, bars, j);
                c.issued = j + 1;
            }
    } else {
        bool ig;
        const int zl = plane_of(c.z0 - 1, g, c.zper, ig);
        load_moments<Codec>(src, g.fstride, c.col + c.plane * (unsigned)zl, p, mn);
    }

    float ppA[8], ppB[8], cA[8], cB[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) ppA[k] = ppB[k] = cA[k] = cB[k] = 0.0f;
    // The window rotates by swapping roles between two register sets, so the
    // march advances two planes per loop trip without register copies.
    bool aborted = false;
    for (int j = 0; j < c.np; j += 2) {
        aborted = K::plane_step(c, g, p, src, dst, tm, stages, bars, ysm, mn, j, ppA, cA, cB);
        if (aborted) break;
        if (j + 1 < c.np) {
            aborted = K::plane_step(c, g, p, src, dst, tm, stages, bars, ysm, mn, j + 1, ppB, cB, cA);
            if (aborted) break;
        }
    }
    if constexpr (TMA) {
        // After a give-up, let every fill already issued land (bounded) before
        // the CTA exits, so no TMA write targets released shared memory.
        if (aborted && c.warp == WROWS - 1 && c.lane == 0) {
            for (int j = c.issued - NSTAGE; j < c.issued; ++j) {
                if (j < 0) continue;
                const uint32_t bar = bars + 8u * (j % NSTAGE), par = (uint32_t)((j / NSTAGE) & 1);
                const long long t0 = clock64();
                while (!mbar_try_wait(bar, par))
                    if (clock64() - t0 > 4000000000LL) break;
            }
        }
    }
}

// ---- host side ------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

template <class Codec>
bool tma_ok(const tslb_s* h) {
    const int E = (int)sizeof(typename Codec::T);
    return ((long long)h->g.nx * E) % 16 == 0 && h->g.nx >= 16 / E && encode_fn() != nullptr;
}

template <class Codec>
bool make_maps(const tslb_s* h, const void* src, TmaMaps* tm) {
    typedef StageLayout<(int)sizeof(typename Codec::T)> SL;
    const int E = (int)sizeof(typename Codec::T);
    const Geometry& g = h->g;
    const CUtensorMapDataType dt = E == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : (h->precision == TSLB_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)NFIELDS};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * E, (cuuint64_t)g.plane * E, (cuuint64_t)g.fstride * E};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const cuuint32_t bmain[4] = {(cuuint32_t)SL::BX, (cuuint32_t)WROWS, 1, 1};
    const cuuint32_t bcol[4] = {(cuuint32_t)SL::XW, (cuuint32_t)WROWS, 1, 1};
    const cuuint32_t brow[4] = {(cuuint32_t)SL::BX, 1, 1, 1};
    const cuuint32_t bcor[4] = {(cuuint32_t)SL::XW, 1, 1, 1};
    EncodeTiledFn fn = encode_fn();
    void* gp = const_cast<void*>(src);
    const cuuint32_t* boxes[4] = {bmain, bcol, brow, bcor};
    CUtensorMap* outs[4] = {&tm->main, &tm->col, &tm->row, &tm->corner};
    for (int k = 0; k < 4; ++k) {
        CUresult r = fn(outs[k], dt, 4, gp, dims, strides, boxes[k], es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

template <class Codec, bool XFREE, bool TMA>
cudaError_t launch_t(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    typedef StageLayout<(int)sizeof(typename Codec::T)> SL;
    auto kern = step_factored_kernel<Codec, XFREE, TMA>;
    const size_t smem = TMA ? SL::SMEM : 128 + YBYTES;
    static bool configured[64] = {};
    const int dev = h->device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SL::SMEM);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    TmaMaps tm;
    memset(&tm, 0, sizeof(tm));
    if (TMA && !make_maps<Codec>(h, src, &tm)) return cudaErrorInvalidValue;
    const Geometry& g = h->g;
    const unsigned bx = (unsigned)((g.nx + XOUT - 1) / XOUT);
    const unsigned by = (unsigned)((g.ny + YOUT - 1) / YOUT);
    const int sms = h->sm_count > 0 ? h->sm_count : 148;
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
    kern<<<dim3(bx, by, bz), NT, smem, h->stream>>>((const typename Codec::T*)src, (typename Codec::T*)dst, g, p,
                                                    zchunk, tm);
    return cudaGetLastError();
}

template <class Codec>
cudaError_t launch_codec(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    const bool xfree = h->g.bc[0] == TSLB_BC_FREESLIP;
    const bool tma = tma_ok<Codec>(h) && h->kernel == TSLB_KERNEL_FACTORED_TMA;
    if (xfree) return tma ? launch_t<Codec, true, true>(h, src, dst, p) : launch_t<Codec, true, false>(h, src, dst, p);
    return tma ? launch_t<Codec, false, true>(h, src, dst, p) : launch_t<Codec, false, false>(h, src, dst, p);
}

}  // namespace

bool factored_supports(const tslb_s* h) {
    // 32-bit node offsets inside a field
    return (long long)h->g.plane * h->g.nz < (1LL << 31);
}

bool factored_uses_tma(const tslb_s* h) {
    switch (h->precision) {
        case TSLB_FP32: return tma_ok<CodecF32>(h) && h->kernel == TSLB_KERNEL_FACTORED_TMA;
        case TSLB_BF16: return tma_ok<CodecBF16>(h) && h->kernel == TSLB_KERNEL_FACTORED_TMA;
        default: return tma_ok<CodecF16>(h) && h->kernel == TSLB_KERNEL_FACTORED_TMA;
    }
}

cudaError_t launch_step_factored(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    switch (h->precision) {
        case TSLB_FP32: return launch_codec<CodecF32>(h, src, dst, p);
        case TSLB_BF16: return launch_codec<CodecBF16>(h, src, dst, p);
        default: return launch_codec<CodecF16>(h, src, dst, p);
    }
}

}  // namespace tslb
