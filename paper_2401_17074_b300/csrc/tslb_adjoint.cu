// Discrete adjoint of the TSLB step with respect to a per-node body force.
//
// The forward step factors into three maps per node (Sec. 2.1-2.2):
//   A(y)  = modes(m(y), F(y))          local, nonlinear (Eq. eqts / Eq. noneqts / Luo force)
//   G(x)  = sum_i T_i A(x - c_i)        linear gather (streaming, Eq. pushLB, and moment sums)
//   m'(x) = finish(G(x))                local, nonlinear (rho, u, Pi^neq from the sums)
// so the adjoint of one step is
//   Gbar(x) = (d finish / d G)^T lambda'(x)
//   Abar(y) = sum_i T_i^T Gbar(y + c_i)                (transpose gather)
//   lambda(y) = (d modes / d m)^T Abar(y),  Fbar(y) += (d modes / d F)^T Abar(y).
// lambda(y) and the state m(y) it pairs with are all the next (earlier) step's
// first map needs, so kernel adj_gather ends with that step's Gbar(y) and the
// lambda array is never stored; adj_seed does the same for the final step.
// The objective is any function J of the final moments, entered through its
// cotangent lambda = dJ/dm (adj_seed_lambda), or J = 1/2 sum rho |u|^2 at the
// final step (adj_seed); the control is a time-constant per-node acceleration
// field.  Segments between the forward
// checkpoints are recomputed with the forward kernel (bitwise identical
// states) and then swept backwards.  Periodic faces, or halfway bounce-back
// walls on the y faces.
#include <cstring>
#include <vector>

#include "tslb_internal.cuh"

#include <nvtx3/nvToolsExt.h>

namespace tslb {
namespace {

template <class Codec>
__device__ __forceinline__ void load_m(const typename Codec::T* __restrict__ src, long long fs, long long idx,
                                       const Physics& p, float m[NFIELDS]) {
    NodeIO<Codec>::load(src, fs, idx, p, m);
}

// Transpose of finish_moments at one node: G = (D0, J, S) -> (drho', u', Pi') with
//   drho' = D0/216, u_a = J_a / r (r = 216 + D0),
//   Pi_aa = (S_aa - J_a^2 / r - D0/3)/216, Pi_ab = (S_ab - J_a J_b / r)/216,
// evaluated at the state m that finish produced.  gb layout: [D0, Jx, Jy, Jz,
// Sxx, Syy, Szz, Sxy, Sxz, Syz].
__device__ __forceinline__ void finish_transpose(const float m[NFIELDS], const float l[NFIELDS], float gb[NFIELDS]) {
    const float u[3] = {m[F_UX], m[F_UY], m[F_UZ]};
    const float inv_r = 1.0f / (216.0f * (1.0f + m[F_DRHO]));
    const float k = 1.0f / 216.0f;
    // lambda_Pi as a symmetric matrix
    const float L[3][3] = {{l[F_PXX], l[F_PXY], l[F_PXZ]}, {l[F_PXY], l[F_PYY], l[F_PYZ]}, {l[F_PXZ], l[F_PYZ], l[F_PZZ]}};
    float gD = l[F_DRHO] * k;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        gD -= u[a] * l[F_UX + a] * inv_r;
        gD += (u[a] * u[a] - 1.0f / 3.0f) * L[a][a] * k;
        float s = 2.0f * u[a] * L[a][a];
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (b != a) s += u[b] * L[a][b];
        gb[1 + a] = l[F_UX + a] * inv_r - s * k;
    }
    gD += (u[0] * u[1] * L[0][1] + u[0] * u[2] * L[0][2] + u[1] * u[2] * L[1][2]) * k;
    gb[0] = gD;
#pragma unroll
    for (int c = 0; c < 6; ++c) gb[4 + c] = l[F_PXX + c] * k;
}

// Gbar layout in its 10 * fs floats: J_a and S_aa are needed together (by
// exactly the directions with c_a != 0), so they are stored as pairs.
//   G0 [fs] | (Jx, Sxx) float2 [fs] | (Jy, Syy) | (Jz, Szz) | Sxy [fs] | Sxz [fs] | Syz [fs]
// gs_off(a): float offset, in units of fs, of scalar array a (G0, Sxy, Sxz,
// Syz); gp_off(a): that of the pair array of axis a.
__host__ __device__ constexpr int gs_off(int a) { return a == 0 ? 0 : 6 + a; }
__host__ __device__ constexpr int gp_off(int a) { return 1 + 2 * a; }
__device__ __forceinline__ void store_gbar(float* __restrict__ G, long long fs, long long n, const float gb[NFIELDS]) {
    G[n] = gb[0];
    reinterpret_cast<float2*>(G + 1 * fs)[n] = make_float2(gb[1], gb[4]);
    reinterpret_cast<float2*>(G + 3 * fs)[n] = make_float2(gb[2], gb[5]);
    reinterpret_cast<float2*>(G + 5 * fs)[n] = make_float2(gb[3], gb[6]);
    G[7 * fs + n] = gb[7];
    G[8 * fs + n] = gb[8];
    G[9 * fs + n] = gb[9];
}

// Final step: lambda = dJ/dm with dJ/d(rho-1) = |u|^2 / 2, dJ/du = rho u,
// dJ/dPi = 0, and the Gbar of the last forward step from it.
template <class Codec>
__global__ void adj_seed(const typename Codec::T* __restrict__ m_end, float* __restrict__ gbar, Geometry g, Physics p) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane * g.nz) return;
    float m[NFIELDS], l[NFIELDS], gb[NFIELDS];
    load_m<Codec>(m_end, g.fstride, n, p, m);
    const float rho = 1.0f + m[F_DRHO];
    l[F_DRHO] = 0.5f * (m[F_UX] * m[F_UX] + m[F_UY] * m[F_UY] + m[F_UZ] * m[F_UZ]);
    l[F_UX] = rho * m[F_UX];
    l[F_UY] = rho * m[F_UY];
    l[F_UZ] = rho * m[F_UZ];
#pragma unroll
    for (int k = 0; k < 6; ++k) l[F_PXX + k] = 0.0f;
    finish_transpose(m, l, gb);
    store_gbar(gbar, g.fstride, n, gb);
}

// Final step with a caller cotangent: lambda = dJ/dm of any objective J of
// the final moments, given as a full-lattice FP64 [10][N] array (rho, u_x,
// u_y, u_z, Pi_xx, Pi_yy, Pi_zz, Pi_xy, Pi_xz, Pi_yz; the rho row is also the
// cotangent of rho - 1), and the Gbar of the last forward step from it.
template <class Codec>
__global__ void adj_seed_lambda(const typename Codec::T* __restrict__ m_end, const double* __restrict__ lam,
                                float* __restrict__ gbar, Geometry g, Physics p, long long fnx, long long fny,
                                long long fN) {
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.plane * g.nz) return;
    const long long xi = n % g.nx, yi = (n / g.nx) % g.ny, zi = n / g.plane;
    const long long node = (xi + g.lo[0]) + fnx * ((yi + g.lo[1]) + fny * (zi + g.lo[2]));
    float m[NFIELDS], l[NFIELDS], gb[NFIELDS];
    load_m<Codec>(m_end, g.fstride, n, p, m);
#pragma unroll
    for (int f = 0; f < NFIELDS; ++f) l[f] = (float)lam[f * fN + node];
    finish_transpose(m, l, gb);
    store_gbar(gbar, g.fstride, n, gb);
}

// Gather blocks: AX x AY x AZ nodes (x fastest), halo tile HX x HY x HZ.
// A tile row holds its HX cells at XOFF .. XOFF + HX - 1 of a PX-float pitch,
// so the AX block columns start on a 16-byte boundary.
constexpr int AX = 32, AY = 4, AZ = 2, AT = AX * AY * AZ;
constexpr int HX = AX + 2, HY = AY + 2, HZ = AZ + 2;
constexpr int PX = 40, XOFF = 3, HC = PX * HY * HZ;
// The tile: the four scalar arrays, float [4][HC], then the three pair arrays,
// float2 [3][HC], in the order of gs_off and gp_off.
constexpr int TILE_FLOATS = 4 * HC + 3 * 2 * HC;
static_assert(TILE_FLOATS == NFIELDS * HC, "ten floats per tile cell");
// Pieces of a tile row in the 16-byte tile load, one thread each: AX / 4 groups
// of four columns and the two halo cells.
constexpr int PIECES = AX / 4 + 2;
static_assert(HY * HZ * PIECES <= AT, "one row piece per thread");
static_assert((XOFF + 1) % 4 == 0 && PX % 4 == 0 && XOFF + HX <= PX, "aligned block columns");

// Transpose gather + transpose of post_modes at the source node y, then the
// Gbar of the preceding step at y (gbar_in belongs to the step m_cur -> m_next,
// gbar_out to the step before it).
// The 27 directions are unrolled, so every coefficient below is a constant:
// a direction loads only the moment sums whose monomial psi_t(c) is nonzero
// (1, 3, 6 or 10 of them for c with 0, 1, 2 or 3 nonzero components), and
// adds only to the modes whose weight w(c) phi_k(c) is nonzero (phi_1(0) = 0).
// WALLS: halfway bounce-back y faces.  A population that the forward step sends
// from y into the wall comes back to y reversed, so a direction c whose target
// y + c lies beyond the wall reads psi(-c) . Gbar(y) instead of
// psi(c) . Gbar(y + c): the thread's own cell, with the odd (J) terms negated.
// VEC: nx is a multiple of 4 and at least AX, so a block's columns, wrapped
// once, are whole aligned groups of 4: a group is one 16-byte copy of each
// scalar array and two of each pair array; the two halo cells are copied
// alone.
template <class Codec, bool VEC, bool WALLS>
__global__ void __launch_bounds__(AT) adj_gather(const float* __restrict__ gbar,
                                                 const typename Codec::T* __restrict__ m_cur,
                                                 float* __restrict__ gbar_out, float* __restrict__ fbar, Geometry g,
                                                 Physics p) {
    // The block's AX x AY x AZ nodes and a one-node halo of Gbar, all ten
    // fields, staged in shared memory with periodic wrap (cp.async copies, all
    // of a thread's in flight at once, no register round trip); the 27
    // directions then read it at constant offsets from the thread's cell.
    __shared__ __align__(16) float tile[TILE_FLOATS];
    float2* const tileP = reinterpret_cast<float2*>(tile + 4 * HC);
    const int tx = threadIdx.x % AX, ty = (threadIdx.x / AX) % AY, tz = threadIdx.x / (AX * AY);
    const int ox = (int)blockIdx.x * AX, oy = (int)blockIdx.y * AY, oz = (int)blockIdx.z * AZ;  // block origin
    const long long fs = g.fstride;
    [[maybe_unused]] const unsigned total = (unsigned)(g.plane * g.nz);
    // launched with programmatic stream serialisation: global memory only
    // after the preceding kernel (a gather or a forward step) has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (VEC) {
        // thread t copies piece t % PIECES of tile row t / PIECES, all ten fields
        const int t = threadIdx.x;
        if (t < HY * HZ * PIECES) {
            const int row = t / PIECES, s = t - row * PIECES;
            const int hy = row % HY, hz = row / HY;
            int gy = oy - 1 + hy, gz = oz - 1 + hz;
            gy = gy < 0 ? gy + g.ny : (gy >= g.ny ? gy - g.ny : gy);
            gz = gz < 0 ? gz + g.nz : (gz >= g.nz ? gz - g.nz : gz);
            // halo cells first (s = 0: x = ox - 1, s = 1: x = ox + AX), then
            // the groups of four columns ox + 4 (s - 2) ...
            const int hx = s == 0 ? 0 : (s == 1 ? HX - 1 : 1 + 4 * (s - 2));
            int gx = ox - 1 + hx;
            gx = gx < 0 ? gx + g.nx : (gx >= g.nx ? gx - g.nx : gx);
            const unsigned gi = (unsigned)gx + (unsigned)g.nx * (unsigned)gy + (unsigned)g.plane * (unsigned)gz;
            const int cell = row * PX + XOFF + hx;
            const unsigned dS = (unsigned)__cvta_generic_to_shared(&tile[cell]);
            const unsigned dP = (unsigned)__cvta_generic_to_shared(&tileP[cell]);
            if (s >= 2) {
                if (TSLB_IN_RANGE(gi + 3, total, p.err)) {
#pragma unroll
                    for (int a = 0; a < 4; ++a)  // four cells of a scalar array: one 16-byte copy
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dS + 4u * a * HC),
                                     "l"(gbar + gs_off(a) * fs + gi) : "memory");
#pragma unroll
                    for (int a = 0; a < 3; ++a) {  // four cells of a pair array: two
                        const float* src = gbar + gp_off(a) * fs + 2ll * gi;
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dP + 8u * a * HC), "l"(src)
                                     : "memory");
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dP + 8u * a * HC + 16u),
                                     "l"(src + 4) : "memory");
                    }
                }
            } else if (TSLB_IN_RANGE(gi, total, p.err)) {
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dS + 4u * a * HC),
                                 "l"(gbar + gs_off(a) * fs + gi) : "memory");
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dP + 8u * a * HC),
                                 "l"(gbar + gp_off(a) * fs + 2ll * gi) : "memory");
            }
        }
    } else {
        // one-step wrap holds for coordinates in [-n, 2n): always in y and z
        // (periodic axes of at least 3 nodes), in x unless the lattice is
        // narrower than about half a block
        const bool xwrap1 = ox + AX < 2 * g.nx;
        for (int c = threadIdx.x; c < HX * HY * HZ; c += AT) {
            const int hx = c % HX, hy = (c / HX) % HY, hz = c / (HX * HY);
            int gx = ox - 1 + hx, gy = oy - 1 + hy, gz = oz - 1 + hz;
            gx = xwrap1 ? (gx < 0 ? gx + g.nx : (gx >= g.nx ? gx - g.nx : gx)) : ((gx % g.nx) + g.nx) % g.nx;
            gy = gy < 0 ? gy + g.ny : (gy >= g.ny ? gy - g.ny : gy);
            gz = gz < 0 ? gz + g.nz : (gz >= g.nz ? gz - g.nz : gz);
            const unsigned gi = (unsigned)gx + (unsigned)g.nx * (unsigned)gy + (unsigned)g.plane * (unsigned)gz;
            const int cell = (hz * HY + hy) * PX + XOFF + hx;
            if (TSLB_IN_RANGE(gi, total, p.err)) {
                const unsigned dS = (unsigned)__cvta_generic_to_shared(&tile[cell]);
                const unsigned dP = (unsigned)__cvta_generic_to_shared(&tileP[cell]);
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dS + 4u * a * HC),
                                 "l"(gbar + gs_off(a) * fs + gi) : "memory");
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dP + 8u * a * HC),
                                 "l"(gbar + gp_off(a) * fs + 2ll * gi) : "memory");
            } else {
#pragma unroll
                for (int a = 0; a < 4; ++a) tile[a * HC + cell] = 0.0f;
#pragma unroll
                for (int a = 0; a < 3; ++a) tileP[a * HC + cell] = make_float2(0.0f, 0.0f);
            }
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    // the node's own state and force load while the tile copies are in flight
    const int px = ox + tx, py = oy + ty, pz = oz + tz;  // this thread's source node
    const bool active = px < g.nx && py < g.ny && pz < g.nz;
    const long long n = active ? (long long)px + (long long)g.nx * py + g.plane * (long long)pz : 0;
    float m[NFIELDS];
    load_m<Codec>(m_cur, g.fstride, n, p, m);
    float F[3] = {p.F[0], p.F[1], p.F[2]};
    if (p.force) {
        const float4 f = reinterpret_cast<const float4*>(p.force)[n];
        F[0] = f.x;
        F[1] = f.y;
        F[2] = f.z;
    }
    const float fb_old[3] = {fbar[n], fbar[fs + n], fbar[2 * fs + n]};
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    if (!active) return;
    const int cc = (tz + 1) * (PX * HY) + (ty + 1) * PX + XOFF + (tx + 1);  // the thread's tile cell
    const bool wall_lo = WALLS && py == 0, wall_hi = WALLS && py == g.ny - 1;  // warp-uniform
    const float* Tc = tile + cc;
    const float2* Pc = tileP + cc;
    float Ab[NMODES];
    float gbv[3][3][3];  // adjoint populations gb(c), [cz + 1][cy + 1][cx + 1]
#pragma unroll
    for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
                // reflected at a y wall: the own cell, J terms negated
                const bool flip = WALLS && ((cy < 0 && wall_lo) || (cy > 0 && wall_hi));
                const int o = flip ? 0 : cz * (PX * HY) + cy * PX + cx;
                const float sj = flip ? -1.0f : 1.0f;
                const float* G = Tc + o;
                const float2* P = Pc + o;
                // adjoint population: psi(c) . Gbar(y + c), nonzero terms only;
                // P[a * HC] = (J_a, S_aa)
                const float2 qx = cx != 0 ? P[0 * HC] : make_float2(0.f, 0.f);
                const float2 qy = cy != 0 ? P[1 * HC] : make_float2(0.f, 0.f);
                const float2 qz = cz != 0 ? P[2 * HC] : make_float2(0.f, 0.f);
                float gb = G[0];
                if (cx != 0) gb = fmaf(sj * cx, qx.x, gb);
                if (cy != 0) gb = fmaf(sj * cy, qy.x, gb);
                if (cz != 0) gb = fmaf(sj * cz, qz.x, gb);
                if (cx != 0) gb += qx.y;
                if (cy != 0) gb += qy.y;
                if (cz != 0) gb += qz.y;
                if (cx != 0 && cy != 0) gb = fmaf((float)(cx * cy), G[1 * HC], gb);
                if (cx != 0 && cz != 0) gb = fmaf((float)(cx * cz), G[2 * HC], gb);
                if (cy != 0 && cz != 0) gb = fmaf((float)(cy * cz), G[3 * HC], gb);
                gbv[cz + 1][cy + 1][cx + 1] = gb;
            }
    // Modes of the adjoint populations, Ab_k = sum_c w(c) phi_k(c) gb(c), one
    // axis at a time: the 1-D weights w phi_0, w phi_1, w phi_2 over c = -1, 0, 1
    // are (1, 4, 1), (-1, 0, 1) and (2, -4, 2).
    float T1[3][3][3];  // [kx][cz][cy]
#pragma unroll
    for (int z = 0; z < 3; ++z)
#pragma unroll
        for (int y = 0; y < 3; ++y) {
            const float a = gbv[z][y][0], b = gbv[z][y][1], c = gbv[z][y][2], e = a + c;
            T1[0][z][y] = fmaf(4.0f, b, e);
            T1[1][z][y] = c - a;
            T1[2][z][y] = fmaf(-4.0f, b, 2.0f * e);
        }
    float T2[3][3][3];  // [kx][ky][cz]
#pragma unroll
    for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int z = 0; z < 3; ++z) {
            const float a = T1[kx][z][0], b = T1[kx][z][1], c = T1[kx][z][2], e = a + c;
            T2[kx][0][z] = fmaf(4.0f, b, e);
            T2[kx][1][z] = c - a;
            T2[kx][2][z] = fmaf(-4.0f, b, 2.0f * e);
        }
#pragma unroll
    for (int k = 0; k < NMODES; ++k) {
        int k1, k2, k3;
        mode_digits(k, k1, k2, k3);
        const float a = T2[k1][k2][0], b = T2[k1][k2][1], c = T2[k1][k2][2];
        Ab[k] = k3 == 0 ? fmaf(4.0f, b, a + c) : (k3 == 1 ? c - a : fmaf(-4.0f, b, 2.0f * (a + c)));
    }
    // transpose of post_modes (u = v, constant or per-node force)
    const float w1 = p.omega1;
    const float rho = 1.0f + m[F_DRHO];
    const float u[3] = {m[F_UX], m[F_UY], m[F_UZ]};
    // Pi as symmetric matrix (stored xx yy zz xy xz yz)
    const float P[3][3] = {{m[F_PXX], m[F_PXY], m[F_PXZ]}, {m[F_PXY], m[F_PYY], m[F_PYZ]}, {m[F_PXZ], m[F_PYZ], m[F_PZZ]}};
    float lr = Ab[M000];
    float lu[3] = {0.f, 0.f, 0.f};
    float lP[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float fb[3];
    // first order: A_a = 3 rho (u_a + F_a)
    const int m1[3] = {M100, M010, M001};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ab = Ab[m1[a]];
        lr += 3.0f * (u[a] + F[a]) * ab;
        lu[a] += 3.0f * rho * ab;
        fb[a] = 3.0f * rho * ab;
    }
    // second order diagonal: A_aa = 1.5 (rho u_a^2 + w1 Pi_aa)
    const int m2d[3] = {M200, M020, M002};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ab = Ab[m2d[a]];
        lr += 1.5f * u[a] * u[a] * ab;
        lu[a] += 3.0f * rho * u[a] * ab;
        lP[a][a] += 1.5f * w1 * ab;
    }
    // second order off-diagonal: A_ab = 9 (rho u_a u_b + w1 Pi_ab)
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    const int m2o[3] = {M110, M101, M011};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int a = pa[q], b = pb[q];
        const float ab = Ab[m2o[q]];
        lr += 9.0f * u[a] * u[b] * ab;
        lu[a] += 9.0f * rho * u[b] * ab;
        lu[b] += 9.0f * rho * u[a] * ab;
        lP[a][b] += 9.0f * w1 * ab;
    }
    // third order A_aab = 4.5 (rho u_a^2 u_b + 2 u_a w1 Pi_ab + u_b w1 Pi_aa)
    const int ta[6] = {0, 0, 1, 1, 2, 2}, tb[6] = {1, 2, 0, 2, 0, 1};
    const int m3[6] = {M210, M201, M120, M021, M102, M012};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int a = ta[q], b = tb[q];
        const float ab = 4.5f * Ab[m3[q]];
        lr += u[a] * u[a] * u[b] * ab;
        lu[a] += (2.0f * rho * u[a] * u[b] + 2.0f * w1 * P[a][b]) * ab;
        lu[b] += (rho * u[a] * u[a] + w1 * P[a][a]) * ab;
        if (a < b) lP[a][b] += 2.0f * u[a] * w1 * ab;
        else lP[b][a] += 2.0f * u[a] * w1 * ab;
        lP[a][a] += u[b] * w1 * ab;
    }
    // A_xyz = 27 (rho u_x u_y u_z + w1 (u_x Pi_yz + u_y Pi_xz + u_z Pi_xy))
    {
        const float ab = 27.0f * Ab[M111];
        lr += u[0] * u[1] * u[2] * ab;
        lu[0] += (rho * u[1] * u[2] + w1 * P[1][2]) * ab;
        lu[1] += (rho * u[0] * u[2] + w1 * P[0][2]) * ab;
        lu[2] += (rho * u[0] * u[1] + w1 * P[0][1]) * ab;
        lP[1][2] += w1 * u[0] * ab;
        lP[0][2] += w1 * u[1] * ab;
        lP[0][1] += w1 * u[2] * ab;
    }
    float l[NFIELDS];
    l[F_DRHO] = lr;
    l[F_UX] = lu[0];
    l[F_UY] = lu[1];
    l[F_UZ] = lu[2];
    l[F_PXX] = lP[0][0];
    l[F_PYY] = lP[1][1];
    l[F_PZZ] = lP[2][2];
    l[F_PXY] = lP[0][1];
    l[F_PXZ] = lP[0][2];
    l[F_PYZ] = lP[1][2];
    float gb[NFIELDS];
    finish_transpose(m, l, gb);
    store_gbar(gbar_out, fs, n, gb);
    fbar[n] = fb_old[0] + fb[0];
    fbar[fs + n] = fb_old[1] + fb[1];
    fbar[2 * fs + n] = fb_old[2] + fb[2];
}

template <class Codec>
cudaError_t adj_launch_all(const tslb_s* h, int which, const void* a, const void* b, float* c, float* d,
                           const Physics& p) {
    const long long total = h->g.plane * h->g.nz;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    typedef typename Codec::T T;
    if (which == 0) {
        if (b) {  // caller cotangent (device FP64 [10][N])
            const long long fnx = h->dims[0], fny = h->dims[1], fN = fnx * fny * h->dims[2];
            adj_seed_lambda<Codec><<<blocks, 256, 0, h->stream>>>((const T*)a, (const double*)b, c, h->g, p, fnx,
                                                                  fny, fN);
        } else {
            adj_seed<Codec><<<blocks, 256, 0, h->stream>>>((const T*)a, c, h->g, p);
        }
    } else {
        const dim3 grid((unsigned)((h->g.nx + AX - 1) / AX), (unsigned)((h->g.ny + AY - 1) / AY),
                        (unsigned)((h->g.nz + AZ - 1) / AZ));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(AT);
        cfg.stream = h->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const bool vec = h->g.nx % 4 == 0 && h->g.nx >= AX, walls = h->bc[2] == TSLB_BC_BOUNCEBACK;
        auto k = vec ? (walls ? adj_gather<Codec, true, true> : adj_gather<Codec, true, false>)
                     : (walls ? adj_gather<Codec, false, true> : adj_gather<Codec, false, false>);
        return cudaLaunchKernelEx(&cfg, k, (const float*)b, (const T*)a, c, d, h->g, p);
    }
    return cudaGetLastError();
}

cudaError_t adj_launch(const tslb_s* h, int which, const void* a, const void* b, float* c, float* d, const Physics& p) {
    switch (h->precision) {
        case TSLB_FP32: return adj_launch_all<CodecF32>(h, which, a, b, c, d, p);
        case TSLB_BF16: return adj_launch_all<CodecBF16>(h, which, a, b, c, d, p);
        default: return adj_launch_all<CodecF16>(h, which, a, b, c, d, p);
    }
}

}  // namespace

// Host driver of the adjoint; error text goes to *msg.  Returns a tslb_status.
// lambda: the caller's cotangent of the final moments (full-lattice FP64
// [10][N], host or device per `where`), or null for J = 1/2 sum rho |u|^2.
int adjoint_run(tslb_s* h, const double* lambda, int64_t nsteps, float* dJdF, int where, std::string* msg) {
    const Geometry& g = h->g;
    const int k = h->checkpoint_every;
    const bool ywalls = h->bc[2] == TSLB_BC_BOUNCEBACK && h->bc[3] == TSLB_BC_BOUNCEBACK;
    for (int f = 0; f < 6; ++f)
        if (h->bc[f] != TSLB_BC_PERIODIC && !(ywalls && (f == 2 || f == 3))) {
            *msg = "the adjoint supports periodic faces and bounce-back walls on the y faces";
            return TSLB_ERR_UNSUPPORTED;
        }
    if (k <= 0) {
        *msg = "create the handle with options.checkpoint_every > 0";
        return TSLB_ERR_STATE;
    }
    if (g.plane * g.nz >= (1LL << 31) || (g.ny + AY - 1) / AY > 65535 || (g.nz + AZ - 1) / AZ > 65535) {
        *msg = "the adjoint supports up to 2^31 - 1 nodes, ny <= 262140 and nz <= 131070";
        return TSLB_ERR_UNSUPPORTED;
    }
    if (nsteps <= 0 || nsteps > h->t || (h->t - nsteps) % k != 0) {
        *msg = "nsteps must be in (0, steps taken] with (steps taken - nsteps) a multiple of checkpoint_every";
        return TSLB_ERR_INVALID;
    }
    if (h->ckpt_valid * k < h->t) {
        *msg = "missing checkpoints";
        return TSLB_ERR_STATE;
    }
    const size_t fs = (size_t)g.fstride;
    const size_t state_bytes = (size_t)NFIELDS * fs * h->elem;
    // workspace, kept in the handle across calls: Gbar of the current step and
    // of the one before, the force gradient, and one recomputed segment (every
    // part a multiple of 512 bytes: fs is padded to 128 nodes)
    const size_t gbar_bytes = sizeof(float) * NFIELDS * fs, fbar_bytes = sizeof(float) * 3 * fs;
    const size_t need = 2 * gbar_bytes + fbar_bytes + state_bytes * (size_t)k;
    // a host cotangent is staged through device memory kept in the handle
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    const size_t lam_bytes = sizeof(double) * NFIELDS * (size_t)fN;
    if (lambda && where == TSLB_HOST && h->adj_lam_bytes < lam_bytes) {
        cudaStreamSynchronize(h->stream);
        if (h->adj_lam) cudaFree(h->adj_lam);
        h->adj_lam = nullptr;
        h->adj_lam_bytes = 0;
        if (cudaMalloc(&h->adj_lam, lam_bytes) != cudaSuccess) {
            h->adj_lam = nullptr;
            *msg = "adjoint cotangent staging allocation failed";
            return TSLB_ERR_ALLOC;
        }
        h->adj_lam_bytes = lam_bytes;
    }
    cudaError_t e = cudaSuccess;
    if (h->adj_ws_bytes < need) {
        cudaStreamSynchronize(h->stream);
        if (h->adj_ws) cudaFree(h->adj_ws);
        h->adj_ws = nullptr;
        h->adj_ws_bytes = 0;
        e = cudaMalloc(&h->adj_ws, need);
        if (e != cudaSuccess) {
            h->adj_ws = nullptr;
            *msg = "adjoint workspace allocation failed";
            return TSLB_ERR_ALLOC;
        }
        h->adj_ws_bytes = need;
    }
    char* ws = static_cast<char*>(h->adj_ws);
    float* gbar[2] = {reinterpret_cast<float*>(ws), reinterpret_cast<float*>(ws + gbar_bytes)};
    float* fbar = reinterpret_cast<float*>(ws + 2 * gbar_bytes);
    char* seg = ws + 2 * gbar_bytes + fbar_bytes;
    auto cleanup = [&]() { cudaStreamSynchronize(h->stream); };
    Physics p = make_physics(h);
    e = cudaMemsetAsync(fbar, 0, sizeof(float) * 3 * fs, h->stream);
    const double* lam_dev = lambda;
    if (lambda && where == TSLB_HOST && e == cudaSuccess) {
        e = cudaMemcpyAsync(h->adj_lam, lambda, lam_bytes, cudaMemcpyHostToDevice, h->stream);
        lam_dev = static_cast<const double*>(h->adj_lam);
    }
    int cur = 0;
    if (e == cudaSuccess) e = adj_launch(h, 0, h->buf[h->cur], lam_dev, gbar[cur], nullptr, p);
    int64_t n_end = h->t;
    const int64_t n_stop = h->t - nsteps;
    while (e == cudaSuccess && n_end > n_stop) {
        const int64_t s = (n_end - 1) / k;
        const int64_t n_beg = s * k;
        const int64_t len = n_end - n_beg;
        nvtxRangePushA("adjoint segment: recompute and backward sweep");
        e = cudaMemcpyAsync(seg, h->ckpts[s], state_bytes, cudaMemcpyDeviceToDevice, h->stream);
        // states n_beg .. n_end - 1 (the gather of step n needs m(n) only)
        for (int64_t j = 0; j + 1 < len && e == cudaSuccess; ++j) {
            Physics pj = p;
            pj.t = n_beg + j;
            pj.sr_key = sr_step_key(h->rounding_seed, pj.t);
            e = launch_step_any(h, seg + j * state_bytes, seg + (j + 1) * state_bytes, pj);
        }
        for (int64_t n = n_end - 1; n >= n_beg && e == cudaSuccess; --n) {
            const char* m_cur = seg + (n - n_beg) * state_bytes;
            e = adj_launch(h, 1, m_cur, gbar[cur], gbar[cur ^ 1], fbar, p);
            cur ^= 1;
        }
        nvtxRangePop();
        n_end = n_beg;
    }
    // scatter the interior gradient into the full-lattice [3][N] output; with
    // y walls its interior rows 1 .. ny - 2 of each z plane, the wall layers 0
    if (e == cudaSuccess) {
        const long long fnx = h->dims[0], fny = h->dims[1];
        const cudaMemcpyKind kind = where == TSLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (!ywalls) {
            for (int a = 0; a < 3 && e == cudaSuccess; ++a)
                e = cudaMemcpyAsync(dJdF + a * fN, fbar + a * fs, sizeof(float) * (size_t)fN, kind, h->stream);
        } else {
            if (where == TSLB_HOST) std::memset(dJdF, 0, sizeof(float) * 3 * (size_t)fN);
            else e = cudaMemsetAsync(dJdF, 0, sizeof(float) * 3 * (size_t)fN, h->stream);
            const size_t row = sizeof(float) * (size_t)g.plane;  // the interior rows of one z plane
            for (int a = 0; a < 3 && e == cudaSuccess; ++a)
                e = cudaMemcpy2DAsync(dJdF + a * fN + fnx * g.lo[1], sizeof(float) * (size_t)(fnx * fny),
                                      fbar + a * fs, row, row, (size_t)g.nz, kind, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cleanup();
    if (e != cudaSuccess) {
        *msg = std::string("adjoint: ") + cudaGetErrorString(e);
        return TSLB_ERR_CUDA;
    }
    return TSLB_OK;
}

}  // namespace tslb
