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
// through shared memory (each warp is a row), then x through warp shuffles
// (lanes are columns).  Halo: lanes 0 and 31 and the first and last row
// recompute the border columns / rows of the tile; the halo rows stop after
// feeding the y exchange.  The z pass starts from the unscaled Hermite
// coefficients with the mode scale factors folded into its fused
// multiply-adds.  The regular stages run on packed FP32x2 instructions over
// pairs of independent groups of the same node (z moments: group pairs; y
// moments: the r = 0, 1 pair of each k1; x pass: output group pairs), which
// halves their issue slots while every value is rounded as in scalar code.
//
// Memory path: each thread copies its column's moments one plane ahead into
// its own shared-memory slots (three cp.async vector copies, L1-cached so the
// halo re-reads of neighbouring tiles hit), reads them back when the plane
// comes up, and stores its node's new moments with three vector stores; the
// y exchange moves four values per shared-memory access.  The exchange is
// synchronised row to row (each warp row waits only for the rows above and
// below, through shared-memory mbarriers) rather than by a CTA barrier, so
// warps drift out of lockstep and the FP-heavy and shared-memory-heavy
// phases of different rows overlap.
//
// Faces: periodic axes wrap; a free-slip face mirrors the 1-D pass (the
// population entering from the wall side is the node's own population leaving
// towards it: specular reflection); a bounce-back y face zeroes the entering
// deviation and adds the reversed populations of the node itself (halfway
// bounce-back), whose moments the warp of the ghost row beyond the wall
// computes in closed form one march step ahead (six y-contracted mode sums),
// so that the wall rows only add them in; inflow / outflow z faces enter the march as ghost planes
// (Eq. neq_final for the inflow, the adjacent layer's moments for the
// outflow, Sec. 3.2).
#pragma once
// (The kernel templates of the sum-factorised step; each storage type is
// instantiated in a translation unit of its own, tslb_step_factored_<type>.cu.)
#include <algorithm>

#include "tslb_internal.cuh"

namespace tslb {
namespace {

constexpr int XOUT = 30;   // output columns per warp (lanes 1..30)
constexpr int WROWS = 18;  // warps per CTA; rows 1..16 are outputs
constexpr int YOUT = WROWS - 2;
constexpr int NT = 32 * WROWS;
// y exchange per thread and buffer: p+ of groups 0-7 (two float4), p- of
// groups 0-7 (two float4), then p+ and p- of group 8 (two floats)
constexpr int YV = 4;  // float4 slots
constexpr int YS = 2;  // float slots
constexpr size_t YBUF = sizeof(float) * (4 * YV + YS) * NT;

// Plane prefetch: every thread copies its column's next-plane moments into its
// own shared-memory slots with cp.async (L1-cached, no registers held while
// the copy is in flight), double-buffered.  Slot regions per buffer: V0, V1
// (16 bytes per thread at FP32, 8 at 16-bit) and V2 (8 / 4 bytes).
template <int E>
struct Prefetch {
    static constexpr int B01 = 4 * E;  // bytes per thread of V0 and of V1
    static constexpr int B2 = 2 * E;   // bytes per thread of V2
    static constexpr size_t BUF = (size_t)(2 * B01 + B2) * NT;
};
// Bounce-back corrections: [2 buffers][2 walls][32 lanes][NCORR] (six
// y-contracted mode sums per lane, padded to eight floats).
constexpr int NCORR = 8;
constexpr size_t CORRBUF = sizeof(float) * 2 * 2 * NCORR * 32;
// Exchange mbarriers: [WROWS rows][2 buffers].
constexpr size_t BARBUF = sizeof(uint64_t) * WROWS * 2;
// With a force field: [2 buffers][NT threads] slots of the node's force
// (the stored float4, 16 bytes each), prefetched with the moments.
constexpr size_t FSLOT = 16;
constexpr size_t FBUF = FSLOT * NT;
template <int E, bool FORCE>
constexpr size_t smem_bytes() {
    return 2 * YBUF + 2 * Prefetch<E>::BUF + CORRBUF + BARBUF + (FORCE ? 2 * FBUF : 0);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Row-to-row synchronisation of the y exchange (one mbarrier per row and
// exchange buffer, arrival count 1): a row arrives (release) after writing its
// slots and waits (acquire) only for the rows above and below.  A row can be
// at most one exchange ahead of its neighbours, so a phase parity identifies
// the exchange unambiguously; the write-after-read on a buffer reused two
// planes later is ordered by the neighbours' arrivals in between, which
// follow their reads.  The bounce-back correction handed from the ghost row
// to the wall row is ordered the same way.
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}
// Arrive only where do_it is set (a predicate instead of a branch).
__device__ __forceinline__ void mbar_arrive_if(uint64_t* bar, bool do_it) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t.reg .pred q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
        "@q mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)), "r"((unsigned)do_it)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after about 2^31 SM clocks, records bit 2 in the
// device status word and stops waiting for the rest of the launch.
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* err, bool& dead) {
    if (mbar_try_wait(bar, parity)) return;
    if (dead) return;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) {
            if (err) atomicOr(err, 2);
            dead = true;
            return;
        }
    }
}

// 1-D populations of a pass: p+, p- and c = a0 - a2 (p0 = 4 c).
struct Pops {
    float pp, pm, c;
};
__device__ __forceinline__ Pops pops3(float a0, float a1, float a2) {
    const float e = fmaf(2.0f, a2, a0);
    return {e + a1, e - a1, a0 - a2};
}
__device__ __forceinline__ Pops pops2(float a0, float a1) { return {a0 + a1, a0 - a1, a0}; }

// Packed FP32x2 arithmetic: two independent mode groups of one node per
// instruction (each lane rounds exactly like the scalar operation).
typedef float2 f2;
__device__ __forceinline__ f2 k2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __ffma2_rn(b, k2(-1.0f), a); }  // a - b, one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
// 1-D populations of two groups: p+, p- and c = a0 - a2.
struct Pops2 {
    f2 pp, pm, c;
};
__device__ __forceinline__ Pops2 pops3(f2 a0, f2 a1, f2 a2) {
    const f2 e = fma2(k2(2.0f), a2, a0);
    return {add2(e, a1), sub2(e, a1), sub2(a0, a2)};
}

// Interior plane stored at march position zs (periodic wrap, inflow / outflow
// ghosts).  On a halo slab the positions -1 and nz are the ghost planes:
// halo = 1 (below) or 2 (above), and the returned plane is 0 of that buffer.
template <bool HALO>
__device__ __forceinline__ int plane_of(int zs, const Geometry& g, bool zper, bool& inflow_ghost, int& halo) {
    inflow_ghost = false;
    halo = 0;
    if (zs < 0) {
        if (zper) return zs + g.nz;
        if (HALO) {
            halo = 1;
            return 0;
        }
        inflow_ghost = true;
        return 0;
    }
    if (zs >= g.nz) {
        if (zper) return zs - g.nz;
        if (HALO) {
            halo = 2;
            return 0;
        }
        return g.nz - 1;  // outflow ghost copies the last layer
    }
    return zs;
}

// Unscaled Hermite coefficients of the post-collision population (see
// post_modes): rho - 1, j = rho (u + F), h2, h3 with P = (1 - omega) Pi;
// (u, F) enter the equilibrium part, (v, Pi) the non-equilibrium part.
struct Herm {
    float drho, jx, jy, jz, xx, yy, zz, xy, xz, yz, xxy, xxz, xyy, yyz, xzz, yzz, xyz;
};
__device__ __forceinline__ Herm hermite(float drho, float ux, float uy, float uz, float vx, float vy, float vz,
                                        const float pi[6], float Fx, float Fy, float Fz, float omega1) {
    Herm h;
    const float rho = 1.0f + drho;
    const float pxx = omega1 * pi[0], pyy = omega1 * pi[1], pzz = omega1 * pi[2];
    const float pxy = omega1 * pi[3], pxz = omega1 * pi[4], pyz = omega1 * pi[5];
    const float rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
    h.drho = drho;
    h.jx = fmaf(rho, Fx, rux);
    h.jy = fmaf(rho, Fy, ruy);
    h.jz = fmaf(rho, Fz, ruz);
    h.xx = fmaf(rux, ux, pxx);
    h.yy = fmaf(ruy, uy, pyy);
    h.zz = fmaf(ruz, uz, pzz);
    const float qxy = rux * uy, qxz = rux * uz, qyz = ruy * uz;
    h.xy = qxy + pxy;
    h.xz = qxz + pxz;
    h.yz = qyz + pyz;
    h.xxy = fmaf(qxy, ux, fmaf(2.0f * vx, pxy, vy * pxx));
    h.xxz = fmaf(qxz, ux, fmaf(2.0f * vx, pxz, vz * pxx));
    h.xyy = fmaf(qxy, uy, fmaf(2.0f * vy, pxy, vx * pyy));
    h.yyz = fmaf(qyz, uy, fmaf(2.0f * vy, pyz, vz * pyy));
    h.xzz = fmaf(qxz, uz, fmaf(2.0f * vz, pxz, vx * pzz));
    h.yzz = fmaf(qyz, uz, fmaf(2.0f * vz, pyz, vy * pzz));
    h.xyz = fmaf(qxy, uz, fmaf(vx, pyz, fmaf(vy, pxz, vz * pxy)));
    return h;
}

// Hermite coefficients in the pair layout of the z pass: scalars drho, h_zz,
// h_xy, j_z, h_xyz and pairs (j_x, j_y), (h_xzz, h_yzz), (h_xz, h_yz),
// (h_xx, h_yy), (h_xxz, h_yyz), (h_xxy, h_xyy).
struct HermP {
    float drho, zz, xy, jz, xyz;
    f2 jxy, h3zz, h2z, h2d, h3z, h3y;
};
__device__ __forceinline__ HermP to_pairs(const Herm& h) {
    HermP q;
    q.drho = h.drho; q.zz = h.zz; q.xy = h.xy; q.jz = h.jz; q.xyz = h.xyz;
    q.jxy = make_float2(h.jx, h.jy);
    q.h3zz = make_float2(h.xzz, h.yzz);
    q.h2z = make_float2(h.xz, h.yz);
    q.h2d = make_float2(h.xx, h.yy);
    q.h3z = make_float2(h.xxz, h.yyz);
    q.h3y = make_float2(h.xxy, h.xyy);
    return q;
}
// Same coefficients where the non-equilibrium velocity is u itself (every
// stored node): with P = (1 - omega) Pi and t_ab = h2_ab + P_ab (= rho u_a u_b
// + 2 P_ab), the third-order terms are h3_aab = u_a t_ab + u_b P_aa and
// h3_xyz = rho u_x u_y u_z + u_x P_yz + u_y P_xz + u_z P_xy.  The x and y
// components run as pairs.
// GUO: Guo forcing (j = rho (u + F/2), h2 += (rho/2)(u F + F u)) instead of
// the Luo term (j = rho (u + F)).
template <bool GUO>
__device__ __forceinline__ HermP hermite_p(float drho, float ux, float uy, float uz, const float pi[6], float Fx,
                                           float Fy, float Fz, float omega1) {
    HermP q;
    const float rho = 1.0f + drho;
    const f2 rho2 = k2(rho), w2 = k2(omega1);
    const f2 Pd = mul2(w2, make_float2(pi[0], pi[1]));   // (P_xx, P_yy)
    const f2 Pzy = mul2(w2, make_float2(pi[2], pi[3]));  // (P_zz, P_xy)
    const f2 Pq = mul2(w2, make_float2(pi[4], pi[5]));   // (P_xz, P_yz)
    const f2 uxy = make_float2(ux, uy), uz2 = k2(uz);
    const f2 ruxy = mul2(rho2, uxy);
    const float ruz = rho * uz;
    q.drho = drho;
    const float jf = GUO ? 0.5f : 1.0f;
    q.jxy = fma2(rho2, make_float2(jf * Fx, jf * Fy), ruxy);
    q.jz = fmaf(rho, jf * Fz, ruz);
    q.h2d = fma2(ruxy, uxy, Pd);
    q.zz = fmaf(ruz, uz, Pzy.x);
    const f2 qz = mul2(ruxy, uz2);  // (rho u_x u_z, rho u_y u_z)
    const float qxy = ruxy.x * uy;
    q.h2z = add2(qz, Pq);
    q.xy = qxy + Pzy.y;
    const f2 tz = add2(q.h2z, Pq);
    const float txy = q.xy + Pzy.y;
    q.h3zz = fma2(uz2, tz, mul2(uxy, k2(Pzy.x)));  // (h_xzz, h_yzz)
    q.h3z = fma2(uxy, tz, mul2(uz2, Pd));          // (h_xxz, h_yyz)
    q.h3y = make_float2(fmaf(ux, txy, uy * Pd.x), fmaf(uy, txy, ux * Pd.y));
    q.xyz = fmaf(qxy, uz, fmaf(ux, Pq.y, fmaf(uy, Pq.x, uz * Pzy.y)));
    if (GUO) {  // after the third-order terms, which take h2 without it
        q.h2d = fma2(ruxy, make_float2(Fx, Fy), q.h2d);
        q.zz = fmaf(ruz, Fz, q.zz);
        q.h2z = fma2(k2(0.5f), fma2(ruxy, k2(Fz), mul2(make_float2(Fx, Fy), k2(ruz))), q.h2z);
        q.xy = fmaf(0.5f, fmaf(ruxy.x, Fy, ruxy.y * Fx), q.xy);
    }
    return q;
}

// z populations of the eight (k1, k2) groups, modes
//   (000, 001, 002) = (drho, 3 j_z, 1.5 h_zz),  (100, 101, 102) = (3 j_x, 9 h_xz, 4.5 h_xzz),
//   (010, 011, 012) = (3 j_y, 9 h_yz, 4.5 h_yzz), (200, 201) = (1.5 h_xx, 4.5 h_xxz),
//   (020, 021) = (1.5 h_yy, 4.5 h_yyz), (110, 111) = (9 h_xy, 27 h_xyz), 210 = 4.5 h_xxy,
//   120 = 4.5 h_xyy, with the scale factors folded into the multiply-adds.
// Pairs of groups in the z pass: G0 = (0, 5), G1 = (1, 2), G2 = (3, 4), G3 = (6, 7).
__device__ __forceinline__ void zpops(const HermP& h, Pops2 P[4]) {
    {
        const f2 e = make_float2(fmaf(3.0f, h.zz, h.drho), 9.0f * h.xy);
        const f2 q = make_float2(h.jz, h.xyz);
        P[0] = {fma2(make_float2(3.0f, 27.0f), q, e), fma2(make_float2(-3.0f, -27.0f), q, e),
                make_float2(fmaf(-1.5f, h.zz, h.drho), e.y)};
    }
    {
        const f2 t = mul2(k2(3.0f), h.jxy), h3 = h.h3zz, h2 = h.h2z;
        const f2 e = fma2(k2(9.0f), h3, t);
        P[1] = {fma2(k2(9.0f), h2, e), fma2(k2(-9.0f), h2, e), fma2(k2(-4.5f), h3, t)};
    }
    {
        const f2 t = mul2(k2(1.5f), h.h2d), q = h.h3z;
        P[2] = {fma2(k2(4.5f), q, t), fma2(k2(-4.5f), q, t), t};
    }
    {
        const f2 t = mul2(k2(4.5f), h.h3y);
        P[3] = {t, t, t};
    }
}

// Body force at stored node idx: the uniform force, or the force field.
__device__ __forceinline__ void load_force(const Physics& p, const Geometry& g, unsigned idx, float& F0, float& F1,
                                           float& F2) {
    F0 = p.F[0];
    F1 = p.F[1];
    F2 = p.F[2];
    if (p.force && TSLB_IN_RANGE(idx, g.plane * g.nz, p.err)) {
        const float4 f = __ldg(reinterpret_cast<const float4*>(p.force) + idx);
        F0 = f.x;
        F1 = f.y;
        F2 = f.z;
    }
}

// Warp-uniform copy of a flag that is equal on all lanes of the warp.  The
// vote lets the compiler see the branch as non-divergent, so the march's
// warp-uniform bookkeeping stays on the uniform datapath.
__device__ __forceinline__ bool uni(bool v) { return __all_sync(0xffffffffu, v); }
// A warp-uniform role flag at its use: voted there (HOIST false), or already
// voted once at set-up (HOIST true).  Both are correct; the step kernel
// hoists the votes for 16-bit storage, where that schedules faster on B300
// (BF16 channel 58.1 -> 60.8 GLUPS), and votes at each use for FP32 storage,
// where hoisting all of them measured slower; the two neighbour-wait flags are
// voted once for every storage type (FP32 +0.85 %).
template <bool HOIST>
__device__ __forceinline__ bool role(bool v) { return HOIST ? v : uni(v); }

// March specialisations by warp role (see Kernel::march).
constexpr int ROLE_ANY = 0, ROLE_PLAIN = 1;

// Per-thread constants of the march.
struct Ctx {
    int tid, lane, warp, x, y, xl, yl;
    unsigned col, plane;
    int z0, z1, np;  // march covers planes z0-1 .. z1 (np of them)
    // out_row .. nee_row, wait_lo, wait_hi are warp-uniform role flags (the
    // wait flags voted at set-up)
    bool zper, ybb, store, out_row, row_lo, row_hi, zero_row, nee_row, xlo_mirror, xhi_mirror, arrive, wait_lo, wait_hi;
    int offLv, offRv, offLs, offRs;  // y-exchange read offsets (float4 / float units, relative to a slot base)
#ifdef TSLB_CHECKED
    int* err;  // device status word, for the index checks
#endif
};

// HALO: a slab of a z-decomposed lattice, whose layers -1 and nz are the
// packed ghost planes p.halo[0] and p.halo[1].
template <class Codec, bool XFREE, bool SPONGE, bool NEEY, bool GUO, bool FORCE, bool HALO>
struct Kernel {
    typedef typename Codec::T T;
    static constexpr bool HOIST = sizeof(T) != 4;
    // the variants launched only without a force field (the plain one is
    // replaced by FORCE when there is one; halo slabs refuse one in tslb_set_force_field)
    static constexpr bool NOFIELD = !FORCE && ((!XFREE && !SPONGE && !NEEY && !GUO) || HALO);

    // One march position j (plane zs = z0 - 1 + j).  ppOld holds p+ of plane
    // zs-2 on entry and p+ of plane zs on exit; cOld holds c of zs-1; cNew
    // receives c of zs.
    typedef Prefetch<(int)sizeof(T)> PF;
    // FORCE: the force slots of buffer PAR, after the mbarriers
    static constexpr size_t FOFF = 2 * PF::BUF + CORRBUF + BARBUF;

    // Start the copies of stored plane zl's moments (march plane j, PAR = j & 1)
    // into prefetch buffer PAR.  The three arrays start fs nodes apart: the
    // moment buffer's field stride, or one plane in a packed ghost plane.
    template <int PAR>
    static __device__ __forceinline__ void prefetch_plane(const Ctx& c, const Geometry& g, const Physics& p,
                                                          const T* __restrict__ src, long long fs, char* pfb,
                                                          int zl) {
        const unsigned n = c.col + c.plane * (unsigned)zl;
        char* b = pfb + PAR * PF::BUF;
        if (TSLB_IN_RANGE(n, g.plane * g.nz, c.err)) {
            cp_async<PF::B01>(smem_u32(b + c.tid * PF::B01), src + (size_t)n * 4);
            cp_async<PF::B01>(smem_u32(b + NT * PF::B01 + c.tid * PF::B01), src + 4 * fs + (size_t)n * 4);
            cp_async<PF::B2>(smem_u32(b + 2 * NT * PF::B01 + c.tid * PF::B2), src + 8 * fs + (size_t)n * 2);
            if (FORCE)
                cp_async<16>(smem_u32(pfb + FOFF + PAR * FBUF + c.tid * FSLOT),
                             reinterpret_cast<const float4*>(p.force) + n);
        }
        cp_async_commit();
    }
    template <int PAR>
    static __device__ __forceinline__ void prefetch(const Ctx& c, const Geometry& g, const Physics& p,
                                                    const T* __restrict__ src, char* pfb, int j) {
        bool ig;
        int hs;
        const int zl = plane_of<HALO>(c.z0 - 1 + j, g, c.zper, ig, hs);
        if (HALO && hs) prefetch_plane<PAR>(c, g, p, static_cast<const T*>(p.halo[hs - 1]), g.plane, pfb, zl);
        else prefetch_plane<PAR>(c, g, p, src, g.fstride, pfb, zl);
    }
    // Body force of the node in prefetch buffer PAR (stored index idx).
    template <int PAR>
    static __device__ __forceinline__ void node_force(const Ctx& c, const Geometry& g, const Physics& p,
                                                      const char* pfb, unsigned idx, float& F0, float& F1, float& F2) {
        if (FORCE) {
            const float* f = reinterpret_cast<const float*>(pfb + FOFF + PAR * FBUF + c.tid * FSLOT);
            F0 = f[0];
            F1 = f[1];
            F2 = f[2];
        } else if (NOFIELD) {
#ifdef TSLB_CHECKED
            // a force field handed to a variant that never reads one
            if (p.force && p.err) atomicOr(p.err, TSLB_ERR_BIT_INDEX);
#endif
            F0 = p.F[0];
            F1 = p.F[1];
            F2 = p.F[2];
        } else {
            load_force(p, g, idx, F0, F1, F2);
        }
    }

    // STEADY: 2 <= j <= np - 3, so the plane and the next one are stored
    // interior planes inside the chunk (no wrap, no ghost, exchange active).
    // ROLE: ROLE_PLAIN for an output row with no wall, ghost or NEE role (its
    // role tests are compile-time constants), ROLE_ANY for the others (tests
    // at run time on the warp's role flags).
    template <int PAR, bool STEADY, int ROLE>
    static __device__ __forceinline__ void plane_step(const Ctx& c, const Geometry& g, const Physics& p,
                                                      const T* __restrict__ src, T* __restrict__ dst, float* ysm,
                                                      char* pfb, float* corr, uint64_t* bars, bool& dead, int j,
                                                      f2 (&ppOld)[4],
                                                      const f2 (&cOld)[4], f2 (&cNew)[4]) {
        const int zs = c.z0 - 1 + j;
        bool inflow_ghost = false;
        int halo = 0;
        const int zl = STEADY ? zs : plane_of<HALO>(zs, g, c.zper, inflow_ghost, halo);
        const unsigned idx = c.col + c.plane * (unsigned)zl;
        // (1 - omega) s_pi of this source plane: uniform, or the sponge layer's
        // value at the plane's lattice z (ghost planes included)
        const int zfull = (!STEADY && c.zper) ? zl : zs + g.lo[2];  // lattice z of the source plane
        const float om_pi = (SPONGE && TSLB_IN_RANGE(zfull, g.nz + 2 * g.lo[2], p.err))
                                ? __ldg(p.omega1_z + zfull) * p.s_pi
                                : p.omega1_pi;
        // next plane's copies go out before this plane's are consumed
        if (STEADY) prefetch_plane<PAR ^ 1>(c, g, p, src, g.fstride, pfb, zs + 1);
        else if (zs < c.z1) prefetch<PAR ^ 1>(c, g, p, src, pfb, j + 1);
        else cp_async_commit();
        cp_async_wait_prev();
        const char* pb = pfb + PAR * PF::BUF;
        const T* v0 = reinterpret_cast<const T*>(pb + c.tid * PF::B01);
        const T* v1 = reinterpret_cast<const T*>(pb + NT * PF::B01 + c.tid * PF::B01);
        const T* v2 = reinterpret_cast<const T*>(pb + 2 * NT * PF::B01 + c.tid * PF::B2);
        // ---- source plane: moments -> Hermite coefficients -> z populations ----
        Pops2 P[4];
        {
            float m[NFIELDS];
            NodeIO<Codec>::decode_smem_rawpi(v0, v1, v2, p, m);
            HermP h;
            if (!STEADY && inflow_ghost) {
                const float uBz = inflow_uz(p, (long long)c.xl + g.lo[0], (long long)c.yl + g.lo[1]);
                h = to_pairs(hermite(m[F_DRHO], 0.f, 0.f, uBz, m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], 0.f, 0.f, 0.f,
                                     om_pi));
            } else if (NEEY && ROLE == ROLE_ANY && role<HOIST>(c.nee_row)) {
                // ghost row beyond an NEE wall: the wall node (whose column is
                // clamped onto the adjacent fluid node) emits f^eq(rho_F, 0) +
                // (1 - omega) f^neq(Pi_F, u_F), Eq. neq_final with u_B = 0
                h = to_pairs(hermite(m[F_DRHO], 0.f, 0.f, 0.f, m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], 0.f, 0.f, 0.f,
                                     om_pi));
            } else {
                float F0, F1, F2;
                node_force<PAR>(c, g, p, pfb, idx, F0, F1, F2);
                h = hermite_p<GUO>(m[F_DRHO], m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], F0, F1, F2, om_pi);
            }
            zpops(h, P);
        }

        if (STEADY || zs >= c.z0 + 1) {
            float* sb = ysm + PAR * (YBUF / sizeof(float));
            float4* sv = reinterpret_cast<float4*>(sb);
            float* ss = sb + 4 * YV * NT;
            // ---- z moments of plane z = zs - 1 (group pairs) ------------------
            f2 Z[4][3];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                Z[i][2] = add2(ppOld[i], P[i].pm);
                Z[i][1] = sub2(ppOld[i], P[i].pm);
                Z[i][0] = fma2(k2(4.0f), cOld[i], Z[i][2]);
            }
            // ---- y pass: groups jj = 3 k1 + r over k2 -----------------------
            // group g of the z pass sits in pair G(g) = {0:(0,x) 1:(1,x) 2:(1,y)
            // 3:(2,x) 4:(2,y) 5:(0,y) 6:(3,x) 7:(3,y)}
            Pops Q[9];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                Q[0 + r] = pops3(Z[0][r].x, Z[1][r].y, Z[2][r].y);  // k1 = 0: k2 = 0, 1, 2 (groups 0, 2, 4)
                Q[3 + r] = pops3(Z[1][r].x, Z[0][r].y, Z[3][r].y);  // k1 = 1 (groups 1, 5, 7)
                Q[6 + r] = pops2(Z[2][r].x, Z[3][r].x);             // k1 = 2 (groups 3, 6)
            }
            // slot order 0 1 3 4 | 6 7 2 5: the (r = 0, r = 1) pair of each k1 is adjacent
            sv[0 * NT + c.tid] = make_float4(Q[0].pp, Q[1].pp, Q[3].pp, Q[4].pp);
            sv[1 * NT + c.tid] = make_float4(Q[6].pp, Q[7].pp, Q[2].pp, Q[5].pp);
            sv[2 * NT + c.tid] = make_float4(Q[0].pm, Q[1].pm, Q[3].pm, Q[4].pm);
            sv[3 * NT + c.tid] = make_float4(Q[6].pm, Q[7].pm, Q[2].pm, Q[5].pm);
            ss[c.tid] = Q[8].pp;
            ss[NT + c.tid] = Q[8].pm;
            __syncwarp();
            mbar_arrive_if(&bars[c.warp * 2 + PAR], c.arrive);
            {
                const unsigned par = (unsigned)((j - 2) >> 1) & 1u;  // phase of this buffer's (j-2)/2-th use
                // plain rows (warps 1 .. WROWS - 2) always have both neighbours
                if (ROLE != ROLE_ANY || c.wait_lo) mbar_wait(&bars[(c.warp - 1) * 2 + PAR], par, p.err, dead);
                if (ROLE != ROLE_ANY || c.wait_hi) mbar_wait(&bars[(c.warp + 1) * 2 + PAR], par, p.err, dead);
            }
            // halo and ghost rows only feed the y exchange (warp-uniform)
            if (ROLE != ROLE_ANY || role<HOIST>(c.out_row)) {
                // L / R: (r = 0, r = 1) pairs per k1 and the r = 2 scalars
                f2 LA[3], RA[3];
                float Ls[3], Rs[3];
                {
                    // plain rows of the variants with periodic x read the rows
                    // below and above (their offsets are constants); the others
                    // may read their own slots on a free-slip wall row
                    constexpr bool COFF = ROLE != ROLE_ANY && !XFREE;
                    const int offLv = COFF ? c.tid - 32 : c.offLv;
                    const int offRv = COFF ? c.tid + 32 : c.offRv;
                    const int offLs = COFF ? c.tid - 32 : c.offLs;
                    const int offRs = COFF ? c.tid + 32 : c.offRs;
                    const float4 l0 = sv[0 * NT + offLv], l1 = sv[1 * NT + offLv];
                    const float4 r0 = sv[2 * NT + offRv], r1 = sv[3 * NT + offRv];
                    LA[0] = make_float2(l0.x, l0.y); LA[1] = make_float2(l0.z, l0.w); LA[2] = make_float2(l1.x, l1.y);
                    RA[0] = make_float2(r0.x, r0.y); RA[1] = make_float2(r0.z, r0.w); RA[2] = make_float2(r1.x, r1.y);
                    Ls[0] = l1.z; Ls[1] = l1.w; Ls[2] = ss[offLs];
                    Rs[0] = r1.z; Rs[1] = r1.w; Rs[2] = ss[NT + offRs];
                }
                // y moments in x-pass pair layout: Y03 = (q,r) groups (0,0) and (0,1),
                // Y14 = (1,0) and (1,1), Y25 = (2,0) and (0,2)
                f2 Y03[3], Y14[3], Y25[3];
#pragma unroll
                for (int k1 = 0; k1 < 3; ++k1) {
                    const f2 cc = make_float2(Q[3 * k1].c, Q[3 * k1 + 1].c);
                    const f2 sLR = add2(LA[k1], RA[k1]);
                    Y03[k1] = fma2(k2(4.0f), cc, sLR);
                    Y14[k1] = sub2(LA[k1], RA[k1]);
                    Y25[k1] = make_float2(LA[k1].x + RA[k1].x, fmaf(4.0f, Q[3 * k1 + 2].c, Ls[k1] + Rs[k1]));
                }
                // ---- x pass: pairs of (q, r) groups over k1 ----------------------
                f2 M0[3], M1[2], M2;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const f2 a0 = k == 0 ? Y03[0] : (k == 1 ? Y14[0] : Y25[0]);
                    const f2 a1 = k == 0 ? Y03[1] : (k == 1 ? Y14[1] : Y25[1]);
                    const f2 a2 = k == 0 ? Y03[2] : (k == 1 ? Y14[2] : Y25[2]);
                    const Pops2 X = pops3(a0, a1, a2);
                    f2 Lx, Rx;
                    Lx.x = __shfl_up_sync(0xffffffffu, X.pp.x, 1);
                    Lx.y = __shfl_up_sync(0xffffffffu, X.pp.y, 1);
                    Rx.x = __shfl_down_sync(0xffffffffu, X.pm.x, 1);
                    Rx.y = __shfl_down_sync(0xffffffffu, X.pm.y, 1);
                    if (XFREE) {
                        if (c.xlo_mirror) Lx = X.pm;
                        if (c.xhi_mirror) Rx = X.pp;
                    }
                    const f2 sLR = add2(Lx, Rx);
                    M0[k] = fma2(k2(4.0f), X.c, sLR);
                    if (k < 2) M1[k] = sub2(Lx, Rx);
                    if (k == 0) M2 = sLR;
                }
                float D0 = M0[0].x;
                float J[3] = {M1[0].x, M0[1].x, M0[0].y};
                float S[6] = {M2.x, M0[2].x, M0[2].y, M1[1].x, M1[0].y, M0[1].y};
                // ---- halfway bounce-back on the wall-adjacent rows ----------
                // The ghost row next to the wall computed the correction for
                // this plane one march step earlier (see bounce_back_correction).
                if (ROLE == ROLE_ANY && c.ybb) {
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        if (!role<HOIST>(side == 0 ? c.row_lo : c.row_hi)) continue;
                        const float* cb = corr + (((PAR ^ 1) * 2 + side) * 32 + c.lane) * NCORR;
                        const float4 b4 = *reinterpret_cast<const float4*>(cb);
                        const float2 b2 = *reinterpret_cast<const float2*>(cb + 4);
                        add_wall_moments(side == 0 ? 1.0f : -1.0f, b4.x, b4.y, b4.z, b4.w, b2.x, b2.y, D0, J, S);
                    }
                }
                float out[NFIELDS];
                if (sizeof(T) == 4) {
                    finish_moments(D0, J, S, out);
                } else {
                    // 16-bit storage: Pi goes straight to storage units (the
                    // 16-bit rounding dominates the single-multiply scaling)
                    const float inv = rcp_refined(216.0f + D0);
                    const float ux = J[0] * inv, uy = J[1] * inv, uz = J[2] * inv;
                    const float d3 = D0 * (1.0f / 3.0f), ps = p.pi_store;
                    out[F_DRHO] = div216(D0);
                    out[F_UX] = ux;
                    out[F_UY] = uy;
                    out[F_UZ] = uz;
                    out[F_PXX] = (S[0] - fmaf(J[0], ux, d3)) * ps;
                    out[F_PYY] = (S[1] - fmaf(J[1], uy, d3)) * ps;
                    out[F_PZZ] = (S[2] - fmaf(J[2], uz, d3)) * ps;
                    out[F_PXY] = (S[3] - J[0] * uy) * ps;
                    out[F_PXZ] = (S[4] - J[0] * uz) * ps;
                    out[F_PYZ] = (S[5] - J[1] * uz) * ps;
                }
                const unsigned oidx = c.col + c.plane * (unsigned)(zs - 1);
                if (GUO) {
                    float G0, G1, G2;
                    load_force(p, g, oidx, G0, G1, G2);
                    guo_finish(out, G0, G1, G2, sizeof(T) == 4 ? 1.0f : p.inv_s_pi);
                }
                // predicated, not branched: only the halo lanes (and lanes
                // beyond the lattice) skip it, and their index is still a
                // valid node (wrapped or clamped column)
                NodeIO<Codec>::store_rawpi_if(dst, g.fstride, oidx, p, out,
                                              c.store && TSLB_IN_RANGE(oidx, g.plane * g.nz, p.err));
            }
        }
        // ---- advance the z window --------------------------------------------
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            ppOld[i] = P[i].pp;
            cNew[i] = P[i].c;
        }
    }

    // The whole z march of one warp: planes 0 and 1 (ghost / wrap, no
    // exchange yet) and the last two or three take the general path; the
    // steady loop in between has none of its tests.  The window rotates by
    // swapping roles between two register sets, so the march advances two
    // planes per loop trip without register copies.
    template <int ROLE>
    static __device__ __forceinline__ void march(const Ctx& c, const Geometry& g, const Physics& p,
                                                 const T* __restrict__ src, T* __restrict__ dst, float* ysm, char* pfb,
                                                 float* corr, uint64_t* bars, bool& dead) {
        f2 ppA[4], ppB[4], cA[4], cB[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) ppA[i] = ppB[i] = cA[i] = cB[i] = k2(0.0f);
        plane_step<0, false, ROLE>(c, g, p, src, dst, ysm, pfb, corr, bars, dead, 0, ppA, cA, cB);
        plane_step<1, false, ROLE>(c, g, p, src, dst, ysm, pfb, corr, bars, dead, 1, ppB, cB, cA);
        int j = 2;
        for (; j + 1 <= c.np - 3; j += 2) {
            plane_step<0, true, ROLE>(c, g, p, src, dst, ysm, pfb, corr, bars, dead, j, ppA, cA, cB);
            plane_step<1, true, ROLE>(c, g, p, src, dst, ysm, pfb, corr, bars, dead, j + 1, ppB, cB, cA);
        }
        for (; j < c.np; j += 2) {
            plane_step<0, false, ROLE>(c, g, p, src, dst, ysm, pfb, corr, bars, dead, j, ppA, cA, cB);
            if (j + 1 < c.np) plane_step<1, false, ROLE>(c, g, p, src, dst, ysm, pfb, corr, bars, dead, j + 1, ppB, cB, cA);
        }
    }

    // The ghost row beyond a bounce-back wall: its exchange slots hold zeros
    // (the deviation entering the wall row from it is zero), written once;
    // each plane it keeps the exchange barriers' rhythm and hands the wall row
    // the closed-form correction of the wall-adjacent node, onto which its
    // column is clamped.  The correction of plane zs, written at march step j
    // into buffer PAR, is read by the wall row at step j + 1 after it has seen
    // this row's arrival of step j + 1 (which follows the write, the warp
    // synchronised); it is overwritten at step j + 2 only after this row has
    // seen the wall row's arrival of step j + 2, which follows that read.
    template <int PAR>
    static __device__ __forceinline__ void ghost_step(const Ctx& c, const Geometry& g, const Physics& p,
                                                      const T* __restrict__ src, char* pfb, float* corr,
                                                      uint64_t* bars, bool& dead, int j) {
        const int zs = c.z0 - 1 + j;
        bool inflow_ghost;
        int halo;
        const int zl = plane_of<HALO>(zs, g, c.zper, inflow_ghost, halo);
        const unsigned idx = c.col + c.plane * (unsigned)zl;
        const int zfull = c.zper ? zl : zs + g.lo[2];
        const float om_pi = (SPONGE && TSLB_IN_RANGE(zfull, g.nz + 2 * g.lo[2], p.err))
                                ? __ldg(p.omega1_z + zfull) * p.s_pi
                                : p.omega1_pi;
        if (zs < c.z1) prefetch<PAR ^ 1>(c, g, p, src, pfb, j + 1);
        else cp_async_commit();
        cp_async_wait_prev();
        if (zs >= c.z0 + 1) {
            __syncwarp();
            mbar_arrive_if(&bars[c.warp * 2 + PAR], c.arrive);
            const unsigned par = (unsigned)((j - 2) >> 1) & 1u;
            if (c.wait_lo) mbar_wait(&bars[(c.warp - 1) * 2 + PAR], par, p.err, dead);
            if (c.wait_hi) mbar_wait(&bars[(c.warp + 1) * 2 + PAR], par, p.err, dead);
        }
        if (zs >= c.z0 && zs < c.z1) {
            const char* pb = pfb + PAR * PF::BUF;
            const T* v0 = reinterpret_cast<const T*>(pb + c.tid * PF::B01);
            const T* v1 = reinterpret_cast<const T*>(pb + NT * PF::B01 + c.tid * PF::B01);
            const T* v2 = reinterpret_cast<const T*>(pb + 2 * NT * PF::B01 + c.tid * PF::B2);
            float m[NFIELDS];
            NodeIO<Codec>::decode_smem_rawpi(v0, v1, v2, p, m);
            float F0, F1, F2;
            node_force<PAR>(c, g, p, pfb, idx, F0, F1, F2);
            bounce_back_correction(m, F0, F1, F2, om_pi, c.y < 0 ? 1.0f : -1.0f,
                                   corr + ((PAR * 2 + (c.y < 0 ? 0 : 1)) * 32 + c.lane) * NCORR);
        }
    }
    static __device__ __forceinline__ void ghost_march(const Ctx& c, const Geometry& g, const Physics& p,
                                                       const T* __restrict__ src, float* ysm, char* pfb, float* corr,
                                                       uint64_t* bars, bool& dead) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float4* sv = reinterpret_cast<float4*>(ysm + b * (YBUF / sizeof(float)));
            float* ss = ysm + b * (YBUF / sizeof(float)) + 4 * YV * NT;
#pragma unroll
            for (int q = 0; q < YV; ++q) sv[q * NT + c.tid] = z4;
            ss[c.tid] = 0.0f;
            ss[NT + c.tid] = 0.0f;
        }
        for (int j = 0; j < c.np; j += 2) {
            ghost_step<0>(c, g, p, src, pfb, corr, bars, dead, j);
            if (j + 1 < c.np) ghost_step<1>(c, g, p, src, pfb, corr, bars, dead, j + 1);
        }
    }

    // Halfway bounce-back at a y wall: the nine populations entering the
    // wall-adjacent node from the wall are its own populations leaving towards
    // the wall, reversed.  By orthogonality of the 1-D basis their moments
    // need only the y-contractions B_kx,kz = A_kx0kz + phi_1(-s) A_kx1kz +
    // 2 A_kx2kz of the post-collision modes at the leaving direction -s, and
    // the 1-D sums 6 (order 0), 2 (c phi_1) and 2 A_0 + 4 A_2 (c^2).
    // s = +1 for the wall below the node, -1 for the wall above.  Writes
    // B00, B10, B01, B20, B02, B11 (one float4 and one float2).
    static __device__ __forceinline__ void bounce_back_correction(const float m[NFIELDS], float F0, float F1, float F2,
                                                                  float omega1, float s, float* out) {
        float Ao[NMODES];
        post_modes(m[F_DRHO], m[F_UX], m[F_UY], m[F_UZ], m[F_UX], m[F_UY], m[F_UZ], &m[F_PXX], F0, F1, F2, omega1, Ao,
                   GUO);
        const float B00 = fmaf(2.0f, Ao[M020], fmaf(-s, Ao[M010], Ao[M000]));
        const float B10 = fmaf(2.0f, Ao[M120], fmaf(-s, Ao[M110], Ao[M100]));
        const float B01 = fmaf(2.0f, Ao[M021], fmaf(-s, Ao[M011], Ao[M001]));
        const float B20 = fmaf(-s, Ao[M210], Ao[M200]);
        const float B02 = fmaf(-s, Ao[M012], Ao[M002]);
        const float B11 = fmaf(-s, Ao[M111], Ao[M101]);
        *reinterpret_cast<float4*>(out) = make_float4(B00, B10, B01, B20);
        *reinterpret_cast<float2*>(out + 4) = make_float2(B02, B11);
    }

    // 216-scaled moment sums of the reversed wall populations (entering y
    // direction s) added to D0, J, S.
    static __device__ __forceinline__ void add_wall_moments(float s, float B00, float B10, float B01, float B20,
                                                            float B02, float B11, float& D0, float J[3], float S[6]) {
        const float b36 = 36.0f * B00, s12 = -12.0f * s;
        D0 += b36;
        J[0] = fmaf(-12.0f, B10, J[0]);
        J[1] = fmaf(s, b36, J[1]);
        J[2] = fmaf(-12.0f, B01, J[2]);
        S[0] = fmaf(12.0f, B00, fmaf(24.0f, B20, S[0]));
        S[1] += b36;
        S[2] = fmaf(12.0f, B00, fmaf(24.0f, B02, S[2]));
        S[3] = fmaf(s12, B10, S[3]);
        S[4] = fmaf(4.0f, B11, S[4]);
        S[5] = fmaf(s12, B01, S[5]);
    }
};

template <class Codec, bool XFREE, bool SPONGE, bool NEEY, bool GUO, bool FORCE, bool HALO>
__global__ void __launch_bounds__(NT, 1)
    step_factored_kernel(const typename Codec::T* __restrict__ src, typename Codec::T* __restrict__ dst, Geometry g,
                         Physics p, int zlo, int zhi, int zchunk) {
    typedef Kernel<Codec, XFREE, SPONGE, NEEY, GUO, FORCE, HALO> K;
    // [2][YBUF] y exchange, [2][PF::BUF] plane prefetch, corrections, mbarriers,
    // and with FORCE [2][FBUF] force slots
    extern __shared__ __align__(16) float ysm[];
    char* pfb = reinterpret_cast<char*>(ysm) + 2 * YBUF;
    float* corr = reinterpret_cast<float*>(pfb + 2 * K::PF::BUF);
    uint64_t* bars = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(corr) + CORRBUF);
    if (threadIdx.x < WROWS * 2) mbar_init(&bars[threadIdx.x], 1);
    __syncthreads();
    bool dead = false;

    Ctx c;
    // Rows to warps.  Warp w issues on SMSP w % 4, so two of the four SMSPs
    // hold five of the 18 warps.  The halo rows 0 and 17 (the lightest:
    // they stop after the y exchange) take warps 0 and 1 on those two, and the
    // rows next to them (the wall rows of a tile at a y wall, the heaviest
    // there) warps 2 and 3 on the SMSPs with four; rows 2 .. 15 take warps
    // 4 .. 17.  Everything below is the row's: c.warp is the row and
    // c.tid = 32 c.warp + lane its slot index.  (Tiles at a bounce-back wall
    // had paced the launch: 3.6 % (FP32) and 5.9 % (BF16) longer than the
    // others with rows on their own warps.)
    {
        const int hw = (int)(threadIdx.x >> 5);
        c.lane = (int)(threadIdx.x & 31);
        c.warp = hw == 0 ? 0 : hw == 1 ? WROWS - 1 : hw == 2 ? 1 : hw == 3 ? WROWS - 2 : hw - 2;
        c.tid = c.warp * 32 + c.lane;
    }
    const int x0 = (int)blockIdx.x * XOUT, y0 = (int)blockIdx.y * YOUT;
    c.x = x0 + c.lane - 1;
    c.y = y0 + c.warp - 1;
    const bool yper = g.bc[2] == TSLB_BC_PERIODIC;
    c.ybb = g.bc[2] == TSLB_BC_BOUNCEBACK;
    const bool yfs = g.bc[2] == TSLB_BC_FREESLIP;
    c.zper = g.bc[4] == TSLB_BC_PERIODIC;
    // Lanes outside the lattice read a wrapped column: on a free-slip x face
    // their values are never used (the boundary lane takes its own mirrored
    // population instead), and distinct columns keep the warp's copies free of
    // repeated addresses, which the copy engine would serialise.
    c.xl = (c.x + g.nx) % g.nx;
    c.yl = yper ? (c.y + g.ny) % g.ny : min(max(c.y, 0), g.ny - 1);
    c.col = (unsigned)c.xl + (unsigned)g.nx * (unsigned)c.yl;
    c.plane = (unsigned)g.plane;
    c.out_row = c.warp >= 1 && c.warp <= YOUT && (yper || (c.y >= 0 && c.y < g.ny));
    c.store = c.lane >= 1 && c.lane <= XOUT && c.x < g.nx && c.warp >= 1 && c.warp <= YOUT && c.y < g.ny;
    c.xlo_mirror = XFREE && c.x == 0;
    c.xhi_mirror = XFREE && c.x == g.nx - 1;
    c.row_lo = c.y == 0;
    c.row_hi = c.y == g.ny - 1;
    c.zero_row = c.ybb && (c.y == -1 || c.y == g.ny);
    c.nee_row = NEEY && (c.y == -1 || c.y == g.ny);
    c.arrive = c.lane == 0 && c.warp != p.drop_row;
    // the neighbour-wait flags are voted once for every storage type
    c.wait_lo = uni(c.warp > 0);
    c.wait_hi = uni(c.warp < WROWS - 1);
    if (K::HOIST) {
        c.out_row = uni(c.out_row);
        c.row_lo = uni(c.row_lo);
        c.row_hi = uni(c.row_hi);
        c.zero_row = uni(c.zero_row);
        c.nee_row = uni(c.nee_row);
    }
    // y-exchange read offsets: the row below / above, or -- on a free-slip wall
    // row -- the node's own value of the opposite population (p- slots sit
    // 2 float4 slots after the p+ slots, the scalar p- one float slot after p+)
    const int below = c.warp > 0 ? c.tid - 32 : c.tid, above = c.warp < WROWS - 1 ? c.tid + 32 : c.tid;
    c.offLv = (yfs && c.row_lo) ? 2 * NT + c.tid : below;
    c.offRv = (yfs && c.row_hi) ? c.tid - 2 * NT : above;
    c.offLs = (yfs && c.row_lo) ? NT + c.tid : below;
    c.offRs = (yfs && c.row_hi) ? c.tid - NT : above;
#ifdef TSLB_CHECKED
    c.err = p.err;
    // every exchange read: float4 slots q * NT + off (q = 0, 1 below, 2, 3
    // above) in [0, YV * NT), float slots off and NT + off in [0, 2 * NT)
    if (!(TSLB_IN_RANGE(c.offLv, YV * NT - NT, p.err) && TSLB_IN_RANGE(2 * NT + c.offRv, YV * NT - NT, p.err) &&
          TSLB_IN_RANGE(c.offLs, 2 * NT, p.err) && TSLB_IN_RANGE(NT + c.offRs, 2 * NT, p.err))) {
        c.offLv = c.offRv = c.offLs = c.offRs = c.tid;
    }
#endif
    // this CTA's z chunk of the launch's layer range [zlo, zhi)
    c.z0 = zlo + (int)blockIdx.z * zchunk;
    c.z1 = min(c.z0 + zchunk, zhi);
    c.np = c.z1 - c.z0 + 2;

    // Launched with programmatic stream serialisation: the set-up above
    // touches only shared memory and parameters and may overlap the end of
    // the preceding step; global memory is read and written only after that
    // step's grid has completed and its writes are visible.  (No early
    // trigger: the next grid starts as this one exits.  Triggering at the
    // start or before the last planes measured slower.)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    K::template prefetch<0>(c, g, p, src, pfb, 0);
    // Output rows without a wall, ghost or NEE role (warp-uniform) run the
    // march with those tests compiled out; the wall, halo, ghost and NEE rows
    // run the general one.  (A third copy for the rows next to a bounce-back
    // wall, with only the wall correction tested, paid off for 16-bit storage
    // before the rows were permuted onto warps; after it, it made the BF16
    // kernel spill 92 bytes instead of 24 and cost 1.2 %.)
    const bool plain = uni(c.warp >= 1 && c.warp <= YOUT && c.out_row && !c.zero_row && !c.nee_row &&
                           !((c.ybb || (!XFREE && yfs)) && (c.row_lo || c.row_hi)));
    // The ghost row beyond a bounce-back wall (warp-uniform) runs a march of
    // its own: in the general one it computed the Hermite and z populations
    // of its node every plane only to write zeros, and the tiles at a wall
    // paced the launch (with the march of its own, and its branches taken out
    // of the general march: BF16 +6 %, FP16 +2.5 %, FP32 +1.2 %).
    if (uni(c.zero_row)) K::ghost_march(c, g, p, src, ysm, pfb, corr, bars, dead);
    else if (plain) K::template march<ROLE_PLAIN>(c, g, p, src, dst, ysm, pfb, corr, bars, dead);
    else K::template march<ROLE_ANY>(c, g, p, src, dst, ysm, pfb, corr, bars, dead);
}

// One step over the layer range [zlo, zhi) of the stored lattice.
template <class Codec, bool XFREE, bool SPONGE, bool NEEY, bool GUO, bool FORCE = false, bool HALO = false>
cudaError_t launch_t(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo, int zhi) {
    auto kern = step_factored_kernel<Codec, XFREE, SPONGE, NEEY, GUO, FORCE, HALO>;
    static bool configured[64] = {};
    const int dev = h->device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    constexpr size_t SMEM = smem_bytes<(int)sizeof(typename Codec::T), FORCE>();
    if (!configured[dev]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    const Geometry& g = h->g;
    const unsigned bx = (unsigned)((g.nx + XOUT - 1) / XOUT);
    const unsigned by = (unsigned)((g.ny + YOUT - 1) / YOUT);
    const int sms = h->sm_count > 0 ? h->sm_count : 148;
    // z chunks: fill whole waves of one CTA per SM while keeping chunks long
    // (each chunk re-reads two extra planes).
    const long long tiles = (long long)bx * by;
    const int nzr = zhi - zlo;
    int best_n = 1;
    double best = 0.0;
    for (int n = 1; n <= 16 && n <= nzr; ++n) {
        const int len = (nzr + n - 1) / n;
        const long long ctas = tiles * n;
        const long long waves = (ctas + sms - 1) / sms;
        const double eff = (double)ctas / (double)(waves * sms) * (double)len / (double)(len + 2);
        if (eff > best + 1e-3) {
            best = eff;
            best_n = n;
        }
    }
    const int zchunk = (nzr + best_n - 1) / best_n;
    const unsigned bz = (unsigned)((nzr + zchunk - 1) / zchunk);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(bx, by, bz);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = h->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, (const typename Codec::T*)src, (typename Codec::T*)dst, g, p, zlo, zhi,
                              zchunk);
}

template <class Codec>
cudaError_t launch_codec(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo, int zhi) {
    const bool xfree = h->g.bc[0] == TSLB_BC_FREESLIP, sponge = p.omega1_z != nullptr;
    // halo slabs: periodic x, periodic or bounce-back y, Luo forcing, constant
    // force (checked at create)
    if (h->g.bc[4] == TSLB_BC_HALO) return launch_t<Codec, false, false, false, false, false, true>(h, src, dst, p, zlo, zhi);
    // Guo forcing comes with periodic x, no sponge and no NEE walls; NEE y walls
    // with periodic x (both checked at create)
    if (p.guo) return launch_t<Codec, false, false, false, true>(h, src, dst, p, zlo, zhi);
    if (h->g.bc[2] == TSLB_BC_NEE_WALL)
        return sponge ? launch_t<Codec, false, true, true, false>(h, src, dst, p, zlo, zhi)
                      : launch_t<Codec, false, false, true, false>(h, src, dst, p, zlo, zhi);
    if (xfree)
        return sponge ? launch_t<Codec, true, true, false, false>(h, src, dst, p, zlo, zhi)
                      : launch_t<Codec, true, false, false, false>(h, src, dst, p, zlo, zhi);
    if (sponge) return launch_t<Codec, false, true, false, false>(h, src, dst, p, zlo, zhi);
    // a force field: its components prefetched with the moments
    return p.force ? launch_t<Codec, false, false, false, false, true>(h, src, dst, p, zlo, zhi)
                   : launch_t<Codec, false, false, false, false>(h, src, dst, p, zlo, zhi);
}

}  // namespace
}  // namespace tslb
