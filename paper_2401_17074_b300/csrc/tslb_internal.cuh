// Internal declarations of the TSLB CUDA library: handle layout, storage
// codecs and the per-node Hermite algebra shared by the step kernels.
//
// Notation follows arXiv 2401.17074, Sec. 2.  The post-collision population
// leaving a node (Eq. LBexp with Eq. eqts and Eq. noneqts, plus the Luo force
// term of Sec. 3.1) is written in the D1Q3 x D1Q3 x D1Q3 tensor-product
// Hermite basis.  With
//     rho = 1 + drho, j = rho (u + F), P = (1 - omega) Pi^neq,
//     h2_ab  = rho u_a u_b + P_ab,
//     h3_abg = rho u_a u_b u_g + u_a P_bg + u_b P_ag + u_g P_ab,
// the deviation from the rest population is
//     f_i - w_i = (1/216) * W(c_i) * sum_k A_k phi_k1(c_ix) phi_k2(c_iy) phi_k3(c_iz),
// with integer 1-D weights W = {1, 4, 1} (= 6 w), integer 1-D Hermite values
// phi_0 = 1, phi_1 = c, phi_2 = 3c^2 - 1 (= 3 (c^2 - cs^2)), and the 17 modes
// the D3Q27 lattice supports up to third order:
//     A_000 = drho,  A_a = 3 j_a,  A_aa = 1.5 h2_aa,  A_ab = 9 h2_ab,
//     A_aab = 4.5 h3_aab,  A_xyz = 27 h3_xyz
// (the xxx-type third-order Hermite polynomials vanish on D3Q27).  Every
// constant in the reconstruction, streaming and moment sums is then an exact
// binary number, so the discrete moment identities hold exactly in FP32 and
// mass and momentum are not rescaled by rounded lattice constants each step;
// the kernels accumulate 216 x the deviation moments and divide once at the end.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "tslb.h"

namespace tslb {

// Field order of the stored moments.
enum Field { F_DRHO = 0, F_UX, F_UY, F_UZ, F_PXX, F_PYY, F_PZZ, F_PXY, F_PXZ, F_PYZ, NFIELDS };

// Mode order of the 17 Hermite coefficients (k1 k2 k3 digits = phi order per axis).
enum Mode {
    M000 = 0,
    M100, M010, M001,
    M200, M020, M002,
    M110, M101, M011,
    M210, M201, M120, M021, M102, M012,
    M111,
    NMODES
};

// Geometry of the stored interior box and its faces, passed by value to kernels.
struct Geometry {
    int nx, ny, nz;        // interior extents (stored)
    int lo[3];             // lattice coordinate of interior index 0 per axis (0 or 1)
    int bc[6];             // face codes
    long long fstride;     // elements between consecutive fields
    long long plane;       // nx * ny
};

struct Physics {
    float omega1;          // 1 - omega
    float F[3];            // constant acceleration
    const float* force;    // per-node acceleration, one float4 (F_x, F_y, F_z, 0) per stored node, or nullptr
    // inflow (z- face)
    long long in_c2[2];
    long long in_d;
    float in_u;
    float in_amp;
    unsigned long long in_seed;
    int in_gauss;          // Gaussian (Box-Muller) instead of uniform inflow noise
    int guo;               // Guo forcing instead of the Luo term
    long long t;           // step index of the state being read
    int* err;              // device status word (nonzero: a kernel gave up a bounded wait)
    int drop_row;          // test hook: warp row of the factored step that withholds its exchange arrival (-1: none)
    // storage scales (16-bit codecs): value = stored * scale
    float s_u, s_pi, inv_s_u, inv_s_pi;
    // (1 - omega) * s_pi, applied to Pi decoded without its storage scale, and
    // inv_s_pi / 216, the factor from the 216-scaled sums to stored Pi
    float omega1_pi, pi_store;
    // key of this step's stochastic-rounding bits (sr_step_key of the seed and
    // t); read by the stochastic-rounding codecs only
    uint32_t sr_key;
    // sponge layer: (1 - omega) per full-lattice z, or nullptr (uniform omega)
    const float* omega1_z;
    // halo slab (TSLB_BC_HALO z faces): the packed ghost planes read as the
    // layers z = -1 (halo[0]) and z = nz (halo[1]); nullptr otherwise
    const void* halo[2];
};

// ---- stochastic rounding ------------------------------------------------------
// Integer hash with low bias: two xorshift-multiply rounds (C. Wellons,
// "Prospecting for hash functions", 2018, the lowbias32 construction).
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
// Key of the random bits used when storing the state at t + 1 (the step that
// reads the state at t); nodes draw mix32(node ^ key) and a second word from it.
__host__ __device__ __forceinline__ uint32_t sr_step_key(unsigned long long seed, long long t) {
    return mix32((uint32_t)seed ^ mix32((uint32_t)t ^ mix32((uint32_t)(seed >> 32) ^ 0x5bd1e995U)));
}

// ---- checked build ------------------------------------------------------------
// With -DTSLB_CHECKED the kernels test each global-memory index (and the step
// kernel its shared-memory exchange offsets) before the access; an index out
// of range sets bit 4 of the device status word and the access is skipped, so
// a wrong index shows as a reported error instead of a memory fault.  The
// product build compiles every test to `true`.
#define TSLB_ERR_BIT_INDEX 4
#ifdef TSLB_CHECKED
__device__ __forceinline__ bool checked_in_range(long long i, long long n, int* err) {
    if (i >= 0 && i < n) return true;
    if (err) atomicOr(err, TSLB_ERR_BIT_INDEX);
    return false;
}
#define TSLB_IN_RANGE(i, n, err) ::tslb::checked_in_range((long long)(i), (long long)(n), (err))
#else
#define TSLB_IN_RANGE(i, n, err) true
#endif

// ---- storage ----------------------------------------------------------------
// One moment buffer holds three arrays of small vectors, one entry per stored
// (interior) node, x fastest:
//     V0 = (u_x, u_y, u_z, rho - 1)        at element 0
//     V1 = (Pi_xx, Pi_yy, Pi_zz, Pi_xy)    at element 4 * fs
//     V2 = (Pi_xz, Pi_yz)                  at element 8 * fs
// (fs = node count padded to 128; 10 * fs elements per buffer).  FP32 storage
// moves 16 + 16 + 8 bytes per node, 16-bit storage 8 + 8 + 4, each warp access
// contiguous.  The 16-bit codecs store u / u_ref and Pi / pi_ref (rho - 1
// unscaled), rounded to nearest even, or -- with stochastic rounding -- u and
// rho - 1 rounded up or down in magnitude with probabilities that make the
// stored value exact in expectation (16 random bits per value).  Those two are
// the conserved moments: each step adds to them increments (a body force of
// 1e-7 per step, say) far below half a 16-bit spacing, which rounding to
// nearest would drop every step.  Pi^neq is rebuilt from the gathered
// populations every step and keeps rounding to nearest.
struct CodecF32 {
    typedef float T;
    static constexpr bool SR = false;
};
struct CodecBF16 {
    static constexpr bool SR = false;
    typedef __nv_bfloat16 T;
    typedef __nv_bfloat162 T2;
    static __device__ __forceinline__ float2 to_f2(T2 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ T2 from_f2(float a, float b) { return __floats2bfloat162_rn(a, b); }
    // Stochastic rounding to BF16 (the upper half of the FP32 pattern): add 16
    // random bits below the kept ones and truncate, which carries into the kept
    // bits with probability (dropped part) / (BF16 spacing), in magnitude.  NaN
    // is kept as it is (adding to its payload could carry into the sign).
    static __device__ __forceinline__ unsigned pack_sr(float a, float b, uint32_t r) {
        const uint32_t ba = __float_as_uint(a), bb = __float_as_uint(b);
        const uint32_t ua = a != a ? ba : ba + (r & 0xffffu);
        const uint32_t ub = b != b ? bb : bb + (r >> 16);
        return __byte_perm(ua, ub, 0x7632);
    }
};
struct CodecF16 {
    static constexpr bool SR = false;
    typedef __half T;
    typedef __half2 T2;
    static __device__ __forceinline__ float2 to_f2(T2 v) { return __half22float2(v); }
    static __device__ __forceinline__ T2 from_f2(float a, float b) { return __floats2half2_rn(a, b); }
    // Stochastic rounding to FP16: add U * (FP16 spacing at |x|) in the
    // direction of x, U = r16 / 2^16, and convert toward zero.  The spacing is
    // 2^(e - 10) for |x| in [2^e, 2^(e+1)), and 2^-24 below the normal range.
    static __device__ __forceinline__ __half sr1(float x, uint32_t r16) {
        const int e = max((int)((__float_as_uint(x) >> 23) & 0xffu) - 127, -14);
        const float ulp = __uint_as_float((uint32_t)(e + 117) << 23);
        return __float2half_rz(fmaf(copysignf((float)r16 * (1.0f / 65536.0f), x), ulp, x));
    }
    static __device__ __forceinline__ unsigned pack_sr(float a, float b, uint32_t r) {
        const __half2 v = __halves2half2(sr1(a, r & 0xffffu), sr1(b, r >> 16));
        return *reinterpret_cast<const unsigned*>(&v);
    }
};
// The same storage formats with stochastic rounding of rho - 1 and u in the step.
struct CodecBF16SR : CodecBF16 {
    static constexpr bool SR = true;
};
struct CodecF16SR : CodecF16 {
    static constexpr bool SR = true;
};

template <class Codec>
struct NodeIO {
    typedef typename Codec::T T;
    typedef typename Codec::T2 T2;
    static __device__ __forceinline__ float2 unpack(unsigned w) { return Codec::to_f2(*reinterpret_cast<const T2*>(&w)); }
    static __device__ __forceinline__ unsigned pack(float a, float b) {
        const T2 v = Codec::from_f2(a, b);
        return *reinterpret_cast<const unsigned*>(&v);
    }
    static __device__ __forceinline__ void load(const T* __restrict__ b, long long fs, long long n, const Physics& p,
                                                float m[NFIELDS]) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(b) + n);
        const uint2 c = __ldg(reinterpret_cast<const uint2*>(b + 4 * fs) + n);
        const unsigned d = __ldg(reinterpret_cast<const unsigned*>(b + 8 * fs) + n);
        const float2 su = make_float2(p.s_u, p.s_u), sp = make_float2(p.s_pi, p.s_pi);
        float2 t = __fmul2_rn(unpack(a.x), su);
        m[F_UX] = t.x;
        m[F_UY] = t.y;
        t = unpack(a.y);
        m[F_UZ] = t.x * p.s_u;
        m[F_DRHO] = t.y;
        t = __fmul2_rn(unpack(c.x), sp);
        m[F_PXX] = t.x;
        m[F_PYY] = t.y;
        t = __fmul2_rn(unpack(c.y), sp);
        m[F_PZZ] = t.x;
        m[F_PXY] = t.y;
        t = __fmul2_rn(unpack(d), sp);
        m[F_PXZ] = t.x;
        m[F_PYZ] = t.y;
    }
    // Decode one node held as V0 / V1 / V2 vectors at v0, v1, v2 (shared memory).
    static __device__ __forceinline__ void decode_smem(const T* v0, const T* v1, const T* v2, const Physics& p,
                                                       float m[NFIELDS]) {
        const uint2 a = *reinterpret_cast<const uint2*>(v0);
        const uint2 c = *reinterpret_cast<const uint2*>(v1);
        const unsigned d = *reinterpret_cast<const unsigned*>(v2);
        const float2 su = make_float2(p.s_u, p.s_u), sp = make_float2(p.s_pi, p.s_pi);
        float2 t = __fmul2_rn(unpack(a.x), su);
        m[F_UX] = t.x;
        m[F_UY] = t.y;
        t = unpack(a.y);
        m[F_UZ] = t.x * p.s_u;
        m[F_DRHO] = t.y;
        t = __fmul2_rn(unpack(c.x), sp);
        m[F_PXX] = t.x;
        m[F_PYY] = t.y;
        t = __fmul2_rn(unpack(c.y), sp);
        m[F_PZZ] = t.x;
        m[F_PXY] = t.y;
        t = __fmul2_rn(unpack(d), sp);
        m[F_PXZ] = t.x;
        m[F_PYZ] = t.y;
    }
    // Same as decode_smem with Pi left in storage units (Pi / pi_ref).
    static __device__ __forceinline__ void decode_smem_rawpi(const T* v0, const T* v1, const T* v2, const Physics& p,
                                                             float m[NFIELDS]) {
        const uint2 a = *reinterpret_cast<const uint2*>(v0);
        const uint2 c = *reinterpret_cast<const uint2*>(v1);
        const unsigned d = *reinterpret_cast<const unsigned*>(v2);
        float2 t = __fmul2_rn(unpack(a.x), make_float2(p.s_u, p.s_u));
        m[F_UX] = t.x;
        m[F_UY] = t.y;
        t = unpack(a.y);
        m[F_UZ] = t.x * p.s_u;
        m[F_DRHO] = t.y;
        t = unpack(c.x);
        m[F_PXX] = t.x;
        m[F_PYY] = t.y;
        t = unpack(c.y);
        m[F_PZZ] = t.x;
        m[F_PXY] = t.y;
        t = unpack(d);
        m[F_PXZ] = t.x;
        m[F_PYZ] = t.y;
    }
    // V0 = (u_x, u_y, u_z, rho - 1) in storage units, rounded to nearest or
    // stochastically (random words drawn from the node index and the step key).
    static __device__ __forceinline__ uint2 v0_word(long long n, const Physics& p, const float m[NFIELDS]) {
        const float iu = p.inv_s_u;
        if (Codec::SR) {
            const uint32_t w0 = mix32((uint32_t)n ^ p.sr_key), w1 = mix32(w0 ^ 0x9e3779b9U);
            return make_uint2(Codec::pack_sr(m[F_UX] * iu, m[F_UY] * iu, w0),
                              Codec::pack_sr(m[F_UZ] * iu, m[F_DRHO], w1));
        }
        return make_uint2(pack(m[F_UX] * iu, m[F_UY] * iu), pack(m[F_UZ] * iu, m[F_DRHO]));
    }
    // Same as store with Pi already in storage units.
    static __device__ __forceinline__ void store_rawpi(T* __restrict__ b, long long fs, long long n, const Physics& p,
                                                       const float m[NFIELDS]) {
        reinterpret_cast<uint2*>(b)[n] = v0_word(n, p, m);
        reinterpret_cast<uint2*>(b + 4 * fs)[n] = make_uint2(pack(m[F_PXX], m[F_PYY]), pack(m[F_PZZ], m[F_PXY]));
        reinterpret_cast<unsigned*>(b + 8 * fs)[n] = pack(m[F_PXZ], m[F_PYZ]);
    }
    // store_rawpi where `pred` holds, as predicated stores (no branch)
    static __device__ __forceinline__ void store_rawpi_if(T* __restrict__ b, long long fs, long long n,
                                                          const Physics& p, const float m[NFIELDS], bool pred) {
        const uint2 w0 = v0_word(n, p, m);
        const uint2 w1 = make_uint2(pack(m[F_PXX], m[F_PYY]), pack(m[F_PZZ], m[F_PXY]));
        const unsigned w2 = pack(m[F_PXZ], m[F_PYZ]);
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
            "@q st.global.v2.b32 [%1], {%4, %5};\n\t"
            "@q st.global.v2.b32 [%2], {%6, %7};\n\t"
            "@q st.global.b32 [%3], %8;\n\t}" ::"r"((unsigned)pred),
            "l"(reinterpret_cast<uint2*>(b) + n), "l"(reinterpret_cast<uint2*>(b + 4 * fs) + n),
            "l"(reinterpret_cast<unsigned*>(b + 8 * fs) + n), "r"(w0.x), "r"(w0.y), "r"(w1.x), "r"(w1.y), "r"(w2)
            : "memory");
    }
    static __device__ __forceinline__ void store(T* __restrict__ b, long long fs, long long n, const Physics& p,
                                                 const float m[NFIELDS]) {
        const float ip = p.inv_s_pi;
        reinterpret_cast<uint2*>(b)[n] = v0_word(n, p, m);
        reinterpret_cast<uint2*>(b + 4 * fs)[n] =
            make_uint2(pack(m[F_PXX] * ip, m[F_PYY] * ip), pack(m[F_PZZ] * ip, m[F_PXY] * ip));
        reinterpret_cast<unsigned*>(b + 8 * fs)[n] = pack(m[F_PXZ] * ip, m[F_PYZ] * ip);
    }
};

template <>
struct NodeIO<CodecF32> {
    static __device__ __forceinline__ void load(const float* __restrict__ b, long long fs, long long n, const Physics&,
                                                float m[NFIELDS]) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(b) + n);
        const float4 c = __ldg(reinterpret_cast<const float4*>(b + 4 * fs) + n);
        const float2 d = __ldg(reinterpret_cast<const float2*>(b + 8 * fs) + n);
        m[F_UX] = a.x;
        m[F_UY] = a.y;
        m[F_UZ] = a.z;
        m[F_DRHO] = a.w;
        m[F_PXX] = c.x;
        m[F_PYY] = c.y;
        m[F_PZZ] = c.z;
        m[F_PXY] = c.w;
        m[F_PXZ] = d.x;
        m[F_PYZ] = d.y;
    }
    static __device__ __forceinline__ void decode_smem(const float* v0, const float* v1, const float* v2,
                                                       const Physics&, float m[NFIELDS]) {
        const float4 a = *reinterpret_cast<const float4*>(v0);
        const float4 c = *reinterpret_cast<const float4*>(v1);
        const float2 d = *reinterpret_cast<const float2*>(v2);
        m[F_UX] = a.x;
        m[F_UY] = a.y;
        m[F_UZ] = a.z;
        m[F_DRHO] = a.w;
        m[F_PXX] = c.x;
        m[F_PYY] = c.y;
        m[F_PZZ] = c.z;
        m[F_PXY] = c.w;
        m[F_PXZ] = d.x;
        m[F_PYZ] = d.y;
    }
    static __device__ __forceinline__ void decode_smem_rawpi(const float* v0, const float* v1, const float* v2,
                                                             const Physics& p, float m[NFIELDS]) {
        decode_smem(v0, v1, v2, p, m);
    }
    static __device__ __forceinline__ void store_rawpi(float* __restrict__ b, long long fs, long long n,
                                                       const Physics& p, const float m[NFIELDS]) {
        store(b, fs, n, p, m);
    }
    // store where `pred` holds, as predicated stores (no branch)
    static __device__ __forceinline__ void store_rawpi_if(float* __restrict__ b, long long fs, long long n,
                                                          const Physics&, const float m[NFIELDS], bool pred) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
            "@q st.global.v4.f32 [%1], {%4, %5, %6, %7};\n\t"
            "@q st.global.v4.f32 [%2], {%8, %9, %10, %11};\n\t"
            "@q st.global.v2.f32 [%3], {%12, %13};\n\t}" ::"r"((unsigned)pred),
            "l"(reinterpret_cast<float4*>(b) + n), "l"(reinterpret_cast<float4*>(b + 4 * fs) + n),
            "l"(reinterpret_cast<float2*>(b + 8 * fs) + n), "f"(m[F_UX]), "f"(m[F_UY]), "f"(m[F_UZ]), "f"(m[F_DRHO]),
            "f"(m[F_PXX]), "f"(m[F_PYY]), "f"(m[F_PZZ]), "f"(m[F_PXY]), "f"(m[F_PXZ]), "f"(m[F_PYZ])
            : "memory");
    }
    static __device__ __forceinline__ void store(float* __restrict__ b, long long fs, long long n, const Physics&,
                                                 const float m[NFIELDS]) {
        reinterpret_cast<float4*>(b)[n] = make_float4(m[F_UX], m[F_UY], m[F_UZ], m[F_DRHO]);
        reinterpret_cast<float4*>(b + 4 * fs)[n] = make_float4(m[F_PXX], m[F_PYY], m[F_PZZ], m[F_PXY]);
        reinterpret_cast<float2*>(b + 8 * fs)[n] = make_float2(m[F_PXZ], m[F_PYZ]);
    }
};

// ---- Hermite algebra -------------------------------------------------------
constexpr float CS2 = 1.0f / 3.0f;

// Mode coefficients (deviation form) of the post-collision population.
// (rho-1, u) enter the equilibrium part, (v, Pi) the non-equilibrium part
// (v = u everywhere except the inflow ghost layer of Eq. neq_final).
// With guo set, (jx_add, jy_add, jz_add) is the acceleration F of Guo's
// forcing: j = rho (u + F/2) and h2 gains (rho/2)(u F + F u); otherwise it is
// the Luo term's F, j = rho (u + F).
__device__ __forceinline__ void post_modes(float drho, float ux, float uy, float uz, float vx, float vy, float vz,
                                           const float pi[6], float jx_add, float jy_add, float jz_add,
                                           float omega1, float A[NMODES], bool guo = false) {
    const float rho = 1.0f + drho;
    const float pxx = omega1 * pi[0], pyy = omega1 * pi[1], pzz = omega1 * pi[2];
    const float pxy = omega1 * pi[3], pxz = omega1 * pi[4], pyz = omega1 * pi[5];
    const float rux = rho * ux, ruy = rho * uy, ruz = rho * uz;
    const float h2xx = fmaf(rux, ux, pxx), h2yy = fmaf(ruy, uy, pyy), h2zz = fmaf(ruz, uz, pzz);
    const float qxy = rux * uy, qxz = rux * uz, qyz = ruy * uz;  // rho u_a u_b
    const float h2xy = qxy + pxy, h2xz = qxz + pxz, h2yz = qyz + pyz;
    // h3_aab = rho u_a u_a u_b + 2 v_a P_ab + v_b P_aa
    const float h3xxy = fmaf(qxy, ux, fmaf(2.0f * vx, pxy, vy * pxx));
    const float h3xxz = fmaf(qxz, ux, fmaf(2.0f * vx, pxz, vz * pxx));
    const float h3xyy = fmaf(qxy, uy, fmaf(2.0f * vy, pxy, vx * pyy));
    const float h3yyz = fmaf(qyz, uy, fmaf(2.0f * vy, pyz, vz * pyy));
    const float h3xzz = fmaf(qxz, uz, fmaf(2.0f * vz, pxz, vx * pzz));
    const float h3yzz = fmaf(qyz, uz, fmaf(2.0f * vz, pyz, vy * pzz));
    const float h3xyz = fmaf(qxy, uz, fmaf(vx, pyz, fmaf(vy, pxz, vz * pxy)));
    const float jf = guo ? 0.5f : 1.0f;
    const float gm = guo ? 1.0f : 0.0f, gh = 0.5f * gm;
    A[M000] = drho;
    A[M100] = 3.0f * fmaf(rho * jf, jx_add, rux);
    A[M010] = 3.0f * fmaf(rho * jf, jy_add, ruy);
    A[M001] = 3.0f * fmaf(rho * jf, jz_add, ruz);
    A[M200] = 1.5f * fmaf(gm * rux, jx_add, h2xx);
    A[M020] = 1.5f * fmaf(gm * ruy, jy_add, h2yy);
    A[M002] = 1.5f * fmaf(gm * ruz, jz_add, h2zz);
    A[M110] = 9.0f * fmaf(gh, fmaf(rux, jy_add, ruy * jx_add), h2xy);
    A[M101] = 9.0f * fmaf(gh, fmaf(rux, jz_add, ruz * jx_add), h2xz);
    A[M011] = 9.0f * fmaf(gh, fmaf(ruy, jz_add, ruz * jy_add), h2yz);
    A[M210] = 4.5f * h3xxy;
    A[M201] = 4.5f * h3xxz;
    A[M120] = 4.5f * h3xyy;
    A[M021] = 4.5f * h3yyz;
    A[M102] = 4.5f * h3xzz;
    A[M012] = 4.5f * h3yzz;
    A[M111] = 27.0f * h3xyz;
}

// Integer 1-D Hermite values and weights of the scaled basis above.
__host__ __device__ __forceinline__ float phi(int k, int c) {
    return k == 0 ? 1.0f : (k == 1 ? (float)c : (float)(3 * c * c - 1));
}
__host__ __device__ __forceinline__ float wgt(int c) { return c == 0 ? 4.0f : 1.0f; }

// Mode digits (k1, k2, k3) per mode index.
__host__ __device__ __forceinline__ void mode_digits(int m, int& k1, int& k2, int& k3) {
    const unsigned char d[NMODES][3] = {
        {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1},
        {0, 1, 1}, {2, 1, 0}, {2, 0, 1}, {1, 2, 0}, {0, 2, 1}, {1, 0, 2}, {0, 1, 2}, {1, 1, 1}};
    k1 = d[m][0]; k2 = d[m][1]; k3 = d[m][2];
}

// 216 x (f_i - w_i) along c = (cx, cy, cz) from the scaled mode coefficients.
__device__ __forceinline__ float pop_dev216(const float A[NMODES], int cx, int cy, int cz) {
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < NMODES; ++m) {
        int k1, k2, k3;
        mode_digits(m, k1, k2, k3);
        s = fmaf(A[m], phi(k1, cx) * phi(k2, cy) * phi(k3, cz), s);
    }
    return wgt(cx) * wgt(cy) * wgt(cz) * s;
}

// New moments from the 216-scaled deviation sums D0 = 216 drho',
// J = 216 j', S_ab = 216 (sum f c_a c_b - cs^2 delta_ab) (Sec. 2.1):
//   drho' = D0/216, u' = J/(216 + D0),
//   Pi'_ab = (S_ab - J_a u'_b - delta_ab D0/3) / 216.
// Division by 216 uses a two-term constant so that it is correctly rounded
// up to ties; the reciprocal of 216 + D0 is refined to about half an ulp.
constexpr float INV216_HI = 0x1.2f684cp-8f;    // fl(1/216)
constexpr float INV216_LO = -0x1.2f684cp-35f;  // 1/216 - INV216_HI (exact)
__device__ __forceinline__ float div216(float x) { return fmaf(x, INV216_HI, x * INV216_LO); }

// 1/r for r = 216 + D0 (a normal number near 216): the hardware approximate
// reciprocal x, then one Newton-Raphson step for f(x) = 1/x - r written with
// fused multiply-adds, e = 1 - r x, x' = x + x e (the iteration analysed in
// P. Markstein, "Computation of elementary functions on the IBM RISC
// System/6000 processor", IBM J. Res. Dev. 34 (1990) 111-119), which squares
// the approximation's relative error; the result is within one ulp of 1/r
// (tests/test_rcp_gpu.py checks that bound and the share of correctly rounded
// results over a sweep of r).
__device__ __forceinline__ float rcp_refined(float r) {
    float i;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(i) : "f"(r));
    const float e = fmaf(-r, i, 1.0f);
    return fmaf(i, e, i);
}

// Guo forcing's part of the new moments (F the acceleration at the node):
// u = J/(216 + D0) + F/2 and Pi^G = (S - J u - delta D0/3)/216 + rho F F/4
// (pi_scale converts Pi to the units out[] holds it in).
__device__ __forceinline__ void guo_finish(float out[NFIELDS], float F0, float F1, float F2, float pi_scale) {
    const float q = 0.25f * (1.0f + out[F_DRHO]) * pi_scale;
    out[F_UX] = fmaf(0.5f, F0, out[F_UX]);
    out[F_UY] = fmaf(0.5f, F1, out[F_UY]);
    out[F_UZ] = fmaf(0.5f, F2, out[F_UZ]);
    out[F_PXX] = fmaf(q * F0, F0, out[F_PXX]);
    out[F_PYY] = fmaf(q * F1, F1, out[F_PYY]);
    out[F_PZZ] = fmaf(q * F2, F2, out[F_PZZ]);
    out[F_PXY] = fmaf(q * F0, F1, out[F_PXY]);
    out[F_PXZ] = fmaf(q * F0, F2, out[F_PXZ]);
    out[F_PYZ] = fmaf(q * F1, F2, out[F_PYZ]);
}

__device__ __forceinline__ void finish_moments(float D0, const float J[3], const float S[6], float out[NFIELDS]) {
    const float inv = rcp_refined(216.0f + D0);
    const float ux = J[0] * inv, uy = J[1] * inv, uz = J[2] * inv;
    const float d3 = D0 * (1.0f / 3.0f);
    out[F_DRHO] = div216(D0);
    out[F_UX] = ux;
    out[F_UY] = uy;
    out[F_UZ] = uz;
    out[F_PXX] = div216(S[0] - fmaf(J[0], ux, d3));
    out[F_PYY] = div216(S[1] - fmaf(J[1], uy, d3));
    out[F_PZZ] = div216(S[2] - fmaf(J[2], uz, d3));
    out[F_PXY] = div216(S[3] - J[0] * uy);
    out[F_PXZ] = div216(S[4] - J[0] * uz);
    out[F_PYZ] = div216(S[5] - J[1] * uz);
}

// Philox4x32-10 (Salmon et al., SC'11) for the inflow noise.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
}

// (1 - omega) of a node at full-lattice z (the sponge layer's table when set).
__device__ __forceinline__ float omega1_at(const Physics& p, int zfull) {
    return p.omega1_z ? __ldg(p.omega1_z + zfull) : p.omega1;
}

// Imposed inflow velocity u_z at lattice column (x, y) for step t.  The draw
// is kept out of line (it runs once per column of the inflow plane) and takes
// its parameters by value, so it leaves the step kernels' register allocation
// alone.
static __device__ __noinline__ float inflow_uz_draw(long long x, long long y, long long c2x, long long c2y, long long d,
                                             long long t, unsigned long long seed, float u_jet, float amp,
                                             int gauss) {
    const long long dx = 2 * x - c2x, dy = 2 * y - c2y;
    if (dx * dx + dy * dy > d * d) return 0.0f;
    uint32_t c[4] = {(uint32_t)x, (uint32_t)y, (uint32_t)t, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    float xi;
    if (gauss) {
        // Box-Muller on the block's first two words: u1 in (0, 1], u2 in [0, 1)
        const float u1 = (float)((c[0] >> 8) + 1u) * (1.0f / 16777216.0f);
        const float u2 = (float)(c[1] >> 8) * (1.0f / 16777216.0f);
        xi = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    } else {
        xi = (float)(c[0] >> 8) * (1.0f / 8388608.0f) - 1.0f;
    }
    return u_jet * (1.0f + amp * xi);
}
__device__ __forceinline__ float inflow_uz(const Physics& p, long long x, long long y) {
    return inflow_uz_draw(x, y, p.in_c2[0], p.in_c2[1], p.in_d, p.t, p.in_seed, p.in_u, p.in_amp, p.in_gauss);
}

}  // namespace tslb

constexpr int NFIELDS_3D = 10;

// ---- handle -----------------------------------------------------------------
struct tslb_s {
    int device = 0;
    int lattice = TSLB_D3Q27;
    int nfields = NFIELDS_3D;  // stored moment fields per node (10, or 6 for D2Q9)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t dims[3] = {0, 0, 0};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    tslb::Geometry g{};
    double tau = 1.0, omega = 1.0;
    double force[3] = {0, 0, 0};
    int precision = TSLB_FP32;
    double u_ref = 0.05, pi_ref = 1e-3;
    int kernel = TSLB_KERNEL_AUTO;
    int sm_count = 148;
    int* dev_err = nullptr;  // device status word of the bounded waits
    int checkpoint_every = 0;
    tslb_inflow inflow{};
    int sponge_width = 0;
    double sponge_k = 0.0;
    float* omega1_z = nullptr;  // sponge layer table, (1 - omega) per full-lattice z
    int forcing = TSLB_FORCING_LUO;
    int rounding = TSLB_ROUND_NEAREST;
    unsigned long long rounding_seed = 0;
    size_t elem = 4;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;
    float* force_field = nullptr;
    int64_t t = 0;
    // diagnostics scratch
    double* diag_part = nullptr;
    int diag_blocks = 0;
    double* diag_host = nullptr;
    // adjoint checkpoints: ckpts[s] holds the moments at step s * checkpoint_every
    // for s < ckpt_valid; the buffers stay allocated for reuse by later runs
    // (tslb_init_moments only resets ckpt_valid) until tslb_destroy
    std::vector<void*> ckpts;
    int64_t ckpt_valid = 0;
    // adjoint workspace (two Gbar arrays, the force gradient, one recomputed
    // segment), kept from the first tslb_adjoint_force_gradient call until
    // tslb_destroy: adj_ws_bytes bytes at adj_ws
    void* adj_ws = nullptr;
    size_t adj_ws_bytes = 0;
    // device copy of a host cotangent for tslb_adjoint (FP64 [10][N]), kept
    // from its first use until tslb_destroy
    void* adj_lam = nullptr;
    size_t adj_lam_bytes = 0;
    // halo slab: two packed ghost planes, [side][V0 plane | V1 plane | V2 plane]
    void* ghost = nullptr;
    // halo slab: the stream of the exports and imports (the handle's own, or
    // the caller's), and events ordering them against the steps: ev_step after
    // each completed step, ev_edges after an open step's edges, ev_halo after
    // the latest import
    cudaStream_t halo_stream = nullptr;
    cudaEvent_t ev_step = nullptr, ev_edges = nullptr, ev_halo = nullptr;
    bool step_open = false;  // between tslb_step_part(EDGES) and (INTERIOR)
    std::string err;
};

// Bytes of one packed plane of a halo slab: ten stored values per interior node of a layer.
inline size_t halo_plane_bytes(const tslb_s* h) { return (size_t)NFIELDS_3D * (size_t)h->g.plane * h->elem; }
// Distance between the two ghost planes in the handle's ghost buffer: the
// packed plane rounded up to 256 bytes, so that the second plane starts on
// the alignment the step kernel's 16-byte plane copies need (a packed plane
// of an odd number of nodes is only 4- or 8-byte aligned at its end).
inline size_t halo_ghost_stride(const tslb_s* h) { return (halo_plane_bytes(h) + 255) / 256 * 256; }

namespace tslb {

// Launchers implemented in the kernel translation units.
cudaError_t launch_step_direct(const tslb_s* h, const void* src, void* dst, const Physics& p);
// D2Q9 variant (tslb_step2d.cu)
cudaError_t launch_step2d(const tslb_s* h, const void* src, void* dst, const Physics& p);
cudaError_t launch_encode2d(const tslb_s* h, const double* rho, const double* u, const double* pi, void* dst);
cudaError_t launch_decode2d(const tslb_s* h, const void* src, double* rho, double* u, double* pi);
cudaError_t launch_diag2d(const tslb_s* h, const void* src, double* out_dev);
cudaError_t launch_step_factored(const tslb_s* h, const void* src, void* dst, const Physics& p);
// The factored step over the stored layers [zlo, zhi) only (a split step).
cudaError_t launch_step_factored_range(const tslb_s* h, const void* src, void* dst, const Physics& p, int zlo,
                                       int zhi);
// The step kernel tslb_step uses for this handle (same choice, bitwise-identical results).
cudaError_t launch_step_any(const tslb_s* h, const void* src, void* dst, const Physics& p);
bool use_factored(const tslb_s* h);
int adjoint_run(tslb_s* h, const double* lambda, int64_t nsteps, float* dJdF, int where, std::string* msg);
bool factored_supports(const tslb_s* h);
cudaError_t launch_encode(const tslb_s* h, const double* rho, const double* u, const double* pi, void* dst,
                          const Physics& p);
cudaError_t launch_decode(const tslb_s* h, const void* src, double* rho, double* u, double* pi, const Physics& p);
// Interleave a planar [3][fstride] force field into one float4 per stored node.
cudaError_t launch_pack_force(const tslb_s* h, const float* planar, float* packed);
cudaError_t launch_diag(const tslb_s* h, const void* src, const Physics& p, double* out_dev);

Physics make_physics(const tslb_s* h);
// Error text reported by tslb_last_error(NULL) on this thread.
void set_global_error(const std::string& msg);

}  // namespace tslb
