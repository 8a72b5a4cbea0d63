// FP64 CPU oracle for the high-order thread-safe lattice Boltzmann (TSLB) step.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
// definition that the CUDA path is checked against.  Only the test-suite,
// the smoke check and the CPU-baseline leg of the benchmark may load it; the
// product path never does.  It shares no source with the CUDA library.
//
// What it computes (arXiv 2401.17074, Sec. 2):
//   * a D3Q27 lattice with cs^2 = 1/3 (Sec. 2, after Eq. lbequil; Fig. d3q27);
//   * third-order Hermite equilibria f^eq (Eq. eqts) and third-order regularised
//     non-equilibrium populations f^neq built from Pi^neq by the Hermite
//     recursion (Eq. noneqts);
//   * the thread-safe update f_i(x+c_i,t+1) = f^eq_i + (1-omega) f^neq_i
//     (Eq. LBexp / Eq. pushLB and the combined update after Eq. noneqts),
//     plus the Luo forcing term rho w_i c_i.F / cs^2 (Sec. 3.1, channel set-up);
//   * macroscopic moments rho, rho u, Pi^neq as sums over the populations
//     (Sec. 2, text after Eq. lbequil, and Sec. 2.1 "10 arrays").
//
// Unlike the CUDA path, which keeps only the 10 moment fields, the oracle
// keeps all 27 populations per node (the paper's "one set of distributions"
// plus moments computed from them) and performs the push-form update node by
// node and direction by direction, with every tensor sum written over the full
// alpha, beta, gamma range.  Boundary handling follows Sec. 2.3 (thread-safe
// non-equilibrium extrapolation, Eq. neq_final) for the inflow face, copies the
// adjacent interior node for the outflow face (Sec. 3.2), and uses halfway
// bounce-back or specular reflection for walls.
//
// Readings of the paper that this file takes (the paper is silent or garbled):
//   R1  D3Q27 weights are the products of the 1-D weights {1/6, 2/3, 1/6};
//       direction index i = (cx+1) + 3(cy+1) + 9(cz+1); opposite = 26 - i.
//   R2  the order-2 term of Eq. noneqts carries w_i and the -cs^2 delta term
//       (as in the order-2 regularised form of Sec. 2.1).
//   R3  a^3_neq = u_a Pi_bg + u_b Pi_ag + u_g Pi_ab (Eq. noneqts), truncated at 3.
//   R4  Pi^neq is stored before collision; (1-omega) is applied on reconstruction.
//   R5  the force F is an acceleration; u = (sum f c)/rho without a half-force shift.
//   R6  the inflow ghost node x_B=(x,y,0) takes rho from x_F=(x,y,1), the imposed
//       velocity u_B for f^eq, and Pi^neq and u of x_F for the Hermite f^neq
//       (Eq. neq_final: all a^n_neq evaluated at x_F).
//   R7  the outflow ghost node (x,y,nz-1) takes the moments of (x,y,nz-2).
//   R8  the jet's sponge layer (Sec. 3.2, viscosity raised towards the exit)
//       is nu(z) = nu (1 + K ((z - z_s)/W)^3) for z > z_s = nz - W, with the
//       exponent taken as +3 (the printed -3 diverges at z_s) and W = nz - z_s
//       as the normalising length (the printed z_end is not defined); every
//       node relaxes with omega(z) = 1 / (1/2 + nu(z)/cs^2) of its own z, ghost
//       layers included.
//   R9  "time-varying Gaussian noise" on the inflow: u_z = u_jet (1 + a xi),
//       xi ~ N(0,1) drawn per column and step by the Box-Muller transform of
//       the same Philox4x32-10 block as the uniform noise:
//       u1 = ((r0 >> 8) + 1) 2^-24 in (0, 1], u2 = (r1 >> 8) 2^-24,
//       xi = sqrt(-2 ln u1) cos(2 pi u2).
//   R11 Guo forcing (an alternative to the Luo term, selected per simulation):
//       velocity u = (sum f c + rho F/2)/rho, stored stress
//       Pi^G = sum f c c - rho u u - rho cs^2 delta + (rho/2)(u F + F u), and
//       f^post = f^eq(rho, u) + (1-omega) f^neq(Pi^G, u) + F_i/2 with Guo's
//       term F_i = w_i rho [(c - u).F / cs^2 + (c.u)(c.F) / cs^4] (the BGK
//       update with (1 - omega/2) F_i, written with the non-equilibrium part
//       f - f^eq + F/2 regularised).  Initial populations from given moments:
//       f^eq + f^neq - F_i/2.  Defined for periodic and wall faces (no ghosts).
//   R10 no-slip walls by the thread-safe non-equilibrium extrapolation
//       (Sec. 2.3, Eq. neq_final with the imposed momentum u_B = 0): the wall
//       sits on the boundary layer y = 0 (or ny-1), whose nodes emit
//       f^eq(rho_F, 0) + (1-omega) Hermite f^neq(Pi^neq, u of x_F) with x_F the
//       adjacent fluid node (rho_B extrapolated from x_F, no body force);
//       populations streamed into the layer are dropped.  Defined for y faces
//       with periodic x and z.
//
// Parity status: every function is pinned by the tests in tests/ (moment
// identities, rest state, conservation, forcing, Taylor-Green and shear-wave
// decay, Poiseuille, free-slip decay, uniform in/outflow, Philox known answers).

#include <complex>
#include <vector>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cstdlib>
#include <limits>
#include <omp.h>

namespace {

typedef std::complex<double> cplx;

const double CS2 = 1.0 / 3.0;
const double CS4 = CS2 * CS2;
const double CS6 = CS4 * CS2;

enum { BC_PERIODIC = 0, BC_BOUNCEBACK = 1, BC_FREESLIP = 2, BC_INFLOW = 3, BC_OUTFLOW = 4, BC_NEE_WALL = 5 };

struct Lattice {
    int c[27][3];
    double w[27];
    Lattice() {
        const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};  // index = c+1 (R1)
        for (int cz = -1; cz <= 1; ++cz)
            for (int cy = -1; cy <= 1; ++cy)
                for (int cx = -1; cx <= 1; ++cx) {
                    int i = (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1);
                    c[i][0] = cx; c[i][1] = cy; c[i][2] = cz;
                    w[i] = w1[cx + 1] * w1[cy + 1] * w1[cz + 1];
                }
    }
    static int opp(int i) { return 26 - i; }
    static int index(int cx, int cy, int cz) { return (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1); }
};
const Lattice L;

inline double delta(int a, int b) { return a == b ? 1.0 : 0.0; }

// Second-order Hermite polynomial H2_ab(c) = c_a c_b - cs^2 delta_ab.
inline double H2(const int* c, int a, int b) { return c[a] * c[b] - CS2 * delta(a, b); }
// Third-order Hermite polynomial
// H3_abg(c) = c_a c_b c_g - cs^2 (c_g delta_ab + c_a delta_bg + c_b delta_ag).
inline double H3(const int* c, int a, int b, int g) {
    return c[a] * c[b] * c[g] - CS2 * (c[g] * delta(a, b) + c[a] * delta(b, g) + c[b] * delta(a, g));
}

// Eq. eqts: third-order equilibrium, full tensor sums.
template <class T>
void feq3(const T& rho, const T u[3], T out[27]) {
    for (int i = 0; i < 27; ++i) {
        const int* c = L.c[i];
        T cu = 0.0, s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < 3; ++a) cu += double(c[a]) * u[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) s2 += H2(c, a, b) * u[a] * u[b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int g = 0; g < 3; ++g) s3 += H3(c, a, b, g) * u[a] * u[b] * u[g];
        out[i] = rho * L.w[i] * (1.0 + cu / CS2 + s2 / (2.0 * CS4) + s3 / (6.0 * CS6));
    }
}

// Eq. noneqts with readings R2, R3: regularised non-equilibrium populations.
template <class T>
void fneq3(const T pi[3][3], const T u[3], T out[27]) {
    for (int i = 0; i < 27; ++i) {
        const int* c = L.c[i];
        T s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) s2 += H2(c, a, b) * pi[a][b];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int g = 0; g < 3; ++g) {
                    T a3 = pi[a][b] * u[g] + u[a] * pi[b][g] + u[b] * pi[a][g];
                    s3 += H3(c, a, b, g) * a3;
                }
        out[i] = L.w[i] * (s2 / (2.0 * CS4) + s3 / (6.0 * CS6));
    }
}

// Moments of a population set (Sec. 2): rho, u = (sum f c)/rho, and
// Pi^neq_ab = sum f c_a c_b - rho u_a u_b - rho cs^2 delta_ab.
template <class T>
void moments(const T* f, T& rho, T u[3], T pi[3][3]) {
    rho = 0.0;
    T j[3] = {0.0, 0.0, 0.0};
    T m2[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m2[a][b] = 0.0;
    for (int i = 0; i < 27; ++i) {
        const int* c = L.c[i];
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += double(c[a]) * f[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) m2[a][b] += double(c[a] * c[b]) * f[i];
    }
    for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) pi[a][b] = m2[a][b] - rho * u[a] * u[b] - rho * CS2 * delta(a, b);
}

// Post-collision populations of one node: Eq. LBexp with the third-order
// Hermite pieces, plus the Luo forcing term rho w_i c_i.F/cs^2 (Sec. 3.1).
// Guo's forcing term F_i = w_i rho [(c - u).F / cs^2 + (c.u)(c.F) / cs^4] (R11).
template <class T>
void guo_term(const T& rho, const T u[3], const T F[3], T out[27]) {
    for (int i = 0; i < 27; ++i) {
        const int* c = L.c[i];
        T cmuF = 0.0, cu = 0.0, cF = 0.0;
        for (int a = 0; a < 3; ++a) {
            cmuF += (double(c[a]) - u[a]) * F[a];
            cu += double(c[a]) * u[a];
            cF += double(c[a]) * F[a];
        }
        out[i] = L.w[i] * rho * (cmuF / CS2 + cu * cF / CS4);
    }
}

template <class T>
void post_collision(const T& rho, const T u[3], const T pi[3][3], double omega, const T F[3],
                    T out[27]) {
    T eq[27], neq[27];
    feq3(rho, u, eq);
    fneq3(pi, u, neq);
    for (int i = 0; i < 27; ++i) {
        const int* c = L.c[i];
        T cF = 0.0;
        for (int a = 0; a < 3; ++a) cF += double(c[a]) * F[a];
        out[i] = eq[i] + (1.0 - omega) * neq[i] + rho * L.w[i] * cF / CS2;
    }
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: 10 rounds of two 32x32->64 multiplies with the
// round keys bumped by the Weyl constants.
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Uniform noise xi in [-1, 1) for inflow column (x, y) at time step t.
// xi = (r0 >> 8) * 2^-23 - 1 is exactly representable in binary32.
double inflow_noise(uint64_t seed, int64_t x, int64_t y, int64_t t) {
    uint32_t ctr[4] = {(uint32_t)x, (uint32_t)y, (uint32_t)t, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    philox4x32_10(ctr, key, r);
    return (double)(r[0] >> 8) * (1.0 / 8388608.0) - 1.0;
}

// Gaussian noise xi ~ N(0,1) for inflow column (x, y) at time step t (R9).
double inflow_noise_gauss(uint64_t seed, int64_t x, int64_t y, int64_t t) {
    uint32_t ctr[4] = {(uint32_t)x, (uint32_t)y, (uint32_t)t, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    philox4x32_10(ctr, key, r);
    const double u1 = (double)((r[0] >> 8) + 1u) * (1.0 / 16777216.0);
    const double u2 = (double)(r[1] >> 8) * (1.0 / 16777216.0);
    const double two_pi = 6.283185307179586476925286766559;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
}

enum { NOISE_UNIFORM = 0, NOISE_GAUSSIAN = 1 };

struct Inflow {
    int64_t center2[2];  // twice the nozzle centre (x, y), in node units
    int64_t diameter;    // nozzle diameter D in node units; inside <=> |2x-cx2|^2+|2y-cy2|^2 <= D^2
    double u_jet;        // imposed axial velocity
    double noise_amp;    // relative noise amplitude a: u_z = u_jet (1 + a xi)
    uint64_t seed;
    int64_t origin[2];   // lattice coordinates of this box's node (0, 0) in a larger lattice
                         // (lets a sub-box reproduce the nozzle and noise of the full one)
    int noise_kind;      // NOISE_UNIFORM (xi ~ U(-1,1)) or NOISE_GAUSSIAN (R9)
};

template <class T>
struct Sim {
    int64_t n[3];
    int bc[6];
    double omega;
    T F[3];
    bool has_field;
    int forcing;  // 0: Luo term, 1: Guo (R11)
    std::vector<T> field;  // [3][N] per-node acceleration
    Inflow inflow;
    int64_t t;
    std::vector<T> f, fnew;  // [node][27]
    int64_t sponge_w;        // sponge layer width W (0: none), R8
    double sponge_k;         // sponge strength K

    // Relaxation rate of a node at lattice z (R8).
    double omega_at(int64_t z) const {
        const int64_t zs = n[2] - sponge_w;
        if (sponge_w <= 0 || z <= zs) return omega;
        const double nu0 = CS2 * (1.0 / omega - 0.5);
        const double r = (double)(z - zs) / (double)sponge_w;
        const double nu = nu0 * (1.0 + sponge_k * r * r * r);
        return 1.0 / (0.5 + nu / CS2);
    }

    int64_t N() const { return n[0] * n[1] * n[2]; }
    int64_t idx(int64_t x, int64_t y, int64_t z) const { return x + n[0] * (y + n[1] * z); }
    int64_t lo(int a) const { return bc[2 * a] == BC_PERIODIC ? 0 : 1; }
    int64_t hi(int a) const { return bc[2 * a + 1] == BC_PERIODIC ? n[a] - 1 : n[a] - 2; }
    bool interior(int64_t x, int64_t y, int64_t z) const {
        return x >= lo(0) && x <= hi(0) && y >= lo(1) && y <= hi(1) && z >= lo(2) && z <= hi(2);
    }
    void force_at(int64_t node, T out[3]) const {
        for (int a = 0; a < 3; ++a) out[a] = has_field ? field[a * N() + node] : F[a];
    }
};

template <class T>
void node_moments(const Sim<T>& s, int64_t node, T& rho, T u[3], T pi[3][3]) {
    moments(&s.f[node * 27], rho, u, pi);
    if (s.forcing == 1) {
        // R11: u += F/2; Pi^G = sum f c c - rho u u - rho cs^2 delta + (rho/2)(u F + F u)
        T F[3], m2[3][3];
        s.force_at(node, F);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) m2[a][b] = pi[a][b] + rho * u[a] * u[b];  // sum f c c - rho cs^2 delta
        for (int a = 0; a < 3; ++a) u[a] = u[a] + 0.5 * F[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                pi[a][b] = m2[a][b] - rho * u[a] * u[b] + 0.5 * rho * (u[a] * F[b] + F[a] * u[b]);
    }
}

// Post-collision populations emitted by source node (x,y,z): an interior node,
// an inflow ghost at z=0 (R6) or an outflow ghost at z=nz-1 (R7).
template <class T>
void source_post(const Sim<T>& s, int64_t x, int64_t y, int64_t z, T out[27]) {
    T rho, u[3], pi[3][3], F[3];
    if (s.bc[4] == BC_INFLOW && z == 0) {
        int64_t nf = s.idx(x, y, 1);
        node_moments(s, nf, rho, u, pi);
        T uB[3] = {0.0, 0.0, 0.0};
        const int64_t X = x + s.inflow.origin[0], Y = y + s.inflow.origin[1];
        int64_t dx = 2 * X - s.inflow.center2[0], dy = 2 * Y - s.inflow.center2[1];
        if (dx * dx + dy * dy <= s.inflow.diameter * s.inflow.diameter) {
            double xi = s.inflow.noise_kind == NOISE_GAUSSIAN ? inflow_noise_gauss(s.inflow.seed, X, Y, s.t)
                                                               : inflow_noise(s.inflow.seed, X, Y, s.t);
            uB[2] = s.inflow.u_jet * (1.0 + s.inflow.noise_amp * xi);
        }
        T eq[27], neq[27];
        feq3(rho, uB, eq);     // imposed velocity, extrapolated density
        fneq3(pi, u, neq);     // Hermite f^neq from x_F (Eq. neq_final)
        const double w = s.omega_at(z);
        for (int i = 0; i < 27; ++i) out[i] = eq[i] + (1.0 - w) * neq[i];
        return;
    }
    const bool nee_lo = s.bc[2] == BC_NEE_WALL && y == 0, nee_hi = s.bc[3] == BC_NEE_WALL && y == s.n[1] - 1;
    if (nee_lo || nee_hi) {  // R10
        node_moments(s, s.idx(x, nee_lo ? 1 : s.n[1] - 2, z), rho, u, pi);
        const T uB[3] = {0.0, 0.0, 0.0};
        T eq[27], neq[27];
        feq3(rho, uB, eq);
        fneq3(pi, u, neq);
        const double w = s.omega_at(z);
        for (int i = 0; i < 27; ++i) out[i] = eq[i] + (1.0 - w) * neq[i];
        return;
    }
    int64_t zs = z;
    if (s.bc[5] == BC_OUTFLOW && z == s.n[2] - 1) zs = s.n[2] - 2;  // zero-gradient copy
    int64_t node = s.idx(x, y, zs);
    node_moments(s, node, rho, u, pi);
    s.force_at(node, F);
    if (s.forcing == 1) {
        T eq[27], neq[27], gF[27];
        feq3(rho, u, eq);
        fneq3(pi, u, neq);
        guo_term(rho, u, F, gF);
        const double w = s.omega_at(z);
        for (int i = 0; i < 27; ++i) out[i] = eq[i] + (1.0 - w) * neq[i] + 0.5 * gF[i];
        return;
    }
    post_collision(rho, u, pi, s.omega_at(z), F, out);
}

// One push-form step (Eq. pushLB): every source emits its 27 post-collision
// populations along c_i; walls reflect them, ghost destinations drop them.
template <class T>
void step_once(Sim<T>& s) {
    const int64_t nz = s.n[2];
    const T nan = std::numeric_limits<double>::quiet_NaN();
    std::fill(s.fnew.begin(), s.fnew.end(), nan);
    const int64_t zlo = (s.bc[4] == BC_INFLOW) ? 0 : s.lo(2);
    const int64_t zhi = (s.bc[5] == BC_OUTFLOW) ? nz - 1 : s.hi(2);
    const int64_t ylo = (s.bc[2] == BC_NEE_WALL) ? 0 : s.lo(1);
    const int64_t yhi = (s.bc[3] == BC_NEE_WALL) ? s.n[1] - 1 : s.hi(1);
    // Sources are independent in push form: each (destination, direction)
    // slot has exactly one source, so (z, y) rows run in parallel.
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t z = zlo; z <= zhi; ++z) {
        for (int64_t y = ylo; y <= yhi; ++y) {
            T post[27];
            for (int64_t x = s.lo(0); x <= s.hi(0); ++x) {
                source_post(s, x, y, z, post);
                const bool ghost = !s.interior(x, y, z);
                const int64_t src[3] = {x, y, z};
                for (int i = 0; i < 27; ++i) {
                    int64_t d[3];
                    int c2[3];
                    bool bounce = false, drop = false;
                    for (int a = 0; a < 3; ++a) {
                        int ca = L.c[i][a];
                        d[a] = src[a] + ca;
                        c2[a] = ca;
                        if (s.bc[2 * a] == BC_PERIODIC) {
                            d[a] = (d[a] + s.n[a]) % s.n[a];
                        } else if (d[a] < s.lo(a) || d[a] > s.hi(a)) {
                            int face = s.bc[2 * a + (d[a] > s.hi(a) ? 1 : 0)];
                            if (face == BC_BOUNCEBACK) bounce = true;
                            else if (face == BC_FREESLIP) { d[a] = src[a]; c2[a] = -ca; }
                            else drop = true;  // into an inflow/outflow ghost layer
                        }
                    }
                    if (ghost) {
                        // ghosts only feed interior nodes (walls reflect as usual)
                        if (bounce || drop || !s.interior(d[0], d[1], d[2])) continue;
                        s.fnew[s.idx(d[0], d[1], d[2]) * 27 + Lattice::index(c2[0], c2[1], c2[2])] = post[i];
                        continue;
                    }
                    if (drop) continue;
                    if (bounce) {
                        s.fnew[s.idx(x, y, z) * 27 + Lattice::opp(i)] = post[i];
                        continue;
                    }
                    s.fnew[s.idx(d[0], d[1], d[2]) * 27 + Lattice::index(c2[0], c2[1], c2[2])] = post[i];
                }
            }
        }
    }
    std::swap(s.f, s.fnew);
    s.t += 1;
}

// Every interior population must have been written by the step (the buffer
// is NaN-filled first), so a gap in the streaming rules shows up as NaN.
template <class T>
int check_filled(const Sim<T>& s) {
    int64_t bad = 0;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : bad)
    for (int64_t z = s.lo(2); z <= s.hi(2); ++z)
        for (int64_t y = s.lo(1); y <= s.hi(1); ++y)
            for (int64_t x = s.lo(0); x <= s.hi(0); ++x)
                for (int i = 0; i < 27; ++i)
                    if (std::isnan(std::real(s.f[s.idx(x, y, z) * 27 + i]))) ++bad;
    return bad ? -1 : 0;
}

template <class T>
int validate_and_init(Sim<T>* s, const int64_t dims[3], double tau, const double F[3], const int bc[6],
                      const Inflow* inflow) {
    if (!(tau > 0.5)) return -2;
    for (int a = 0; a < 3; ++a) {
        s->n[a] = dims[a];
        s->bc[2 * a] = bc[2 * a];
        s->bc[2 * a + 1] = bc[2 * a + 1];
        bool per_lo = bc[2 * a] == BC_PERIODIC, per_hi = bc[2 * a + 1] == BC_PERIODIC;
        if (per_lo != per_hi) return -3;
        if (dims[a] < (per_lo ? 3 : 4)) return -4;
    }
    // inflow only on the z- face, outflow only on the z+ face, and as a pair
    for (int f = 0; f < 6; ++f) {
        if (bc[f] == BC_INFLOW && f != 4) return -3;
        if (bc[f] == BC_OUTFLOW && f != 5) return -3;
        if (bc[f] < BC_PERIODIC || bc[f] > BC_NEE_WALL) return -3;
        if (bc[f] == BC_NEE_WALL && f != 2 && f != 3) return -3;
    }
    if ((bc[2] == BC_NEE_WALL || bc[3] == BC_NEE_WALL) && (bc[0] != BC_PERIODIC || bc[4] != BC_PERIODIC)) return -3;
    if ((bc[4] == BC_INFLOW) != (bc[5] == BC_OUTFLOW)) return -3;
    s->omega = 1.0 / tau;
    for (int a = 0; a < 3; ++a) s->F[a] = F ? F[a] : 0.0;
    s->has_field = false;
    std::memset(&s->inflow, 0, sizeof(Inflow));
    if (inflow) s->inflow = *inflow;
    s->t = 0;
    s->sponge_w = 0;
    s->sponge_k = 0.0;
    s->forcing = 0;
    s->f.assign(s->N() * 27, T(0.0));
    s->fnew.assign(s->N() * 27, T(0.0));
    return 0;
}

// Initial populations: f = f^eq3(rho,u) + f^neq3(Pi,u) (the post-collision
// form with omega = 0 and no force); for interior nodes only.
template <class T>
void init_from_moments(Sim<T>* s, const T* rho, const T* u, const T* pi) {
    const int64_t N = s->N();
    for (int64_t z = s->lo(2); z <= s->hi(2); ++z)
        for (int64_t y = s->lo(1); y <= s->hi(1); ++y)
            for (int64_t x = s->lo(0); x <= s->hi(0); ++x) {
                int64_t node = s->idx(x, y, z);
                T r = rho[node];
                T uu[3] = {u[node], u[N + node], u[2 * N + node]};
                T p[3][3];
                const int ord[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
                for (int k = 0; k < 6; ++k) {
                    T v = pi ? pi[k * N + node] : T(0.0);
                    p[ord[k][0]][ord[k][1]] = v;
                    p[ord[k][1]][ord[k][0]] = v;
                }
                T eq[27], neq[27];
                feq3(r, uu, eq);
                fneq3(p, uu, neq);
                for (int i = 0; i < 27; ++i) s->f[node * 27 + i] = eq[i] + neq[i];
                if (s->forcing == 1) {  // R11: the populations whose moments are the given state
                    T F[3], gF[27];
                    s->force_at(node, F);
                    guo_term(r, uu, F, gF);
                    for (int i = 0; i < 27; ++i) s->f[node * 27 + i] -= 0.5 * gF[i];
                }
            }
    s->t = 0;
}

// Full-lattice moments; non-interior nodes report the rest state.
template <class T>
void get_moments(const Sim<T>* s, T* rho, T* u, T* pi) {
    const int64_t N = s->N();
    for (int64_t z = 0; z < s->n[2]; ++z)
        for (int64_t y = 0; y < s->n[1]; ++y)
            for (int64_t x = 0; x < s->n[0]; ++x) {
                int64_t node = s->idx(x, y, z);
                T r = 1.0, uu[3] = {0.0, 0.0, 0.0}, p[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) p[a][b] = 0.0;
                if (s->interior(x, y, z)) node_moments(*s, node, r, uu, p);
                if (rho) rho[node] = r;
                if (u)
                    for (int a = 0; a < 3; ++a) u[a * N + node] = uu[a];
                const int ord[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
                if (pi)
                    for (int k = 0; k < 6; ++k) pi[k * N + node] = p[ord[k][0]][ord[k][1]];
            }
}

}  // namespace

extern "C" {

// ---- per-node primitives (for the identity pins) -------------------------
void orc_lattice(int* c /*27x3*/, double* w /*27*/) {
    for (int i = 0; i < 27; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
        w[i] = L.w[i];
    }
}
void orc_feq3(double rho, const double* u, double* out) { feq3<double>(rho, u, out); }
void orc_fneq3(const double* pi6, const double* u, double* out) {
    double p[3][3] = {{pi6[0], pi6[3], pi6[4]}, {pi6[3], pi6[1], pi6[5]}, {pi6[4], pi6[5], pi6[2]}};
    fneq3<double>(p, u, out);
}
void orc_post(double rho, const double* u, const double* pi6, double omega, const double* F, double* out) {
    double p[3][3] = {{pi6[0], pi6[3], pi6[4]}, {pi6[3], pi6[1], pi6[5]}, {pi6[4], pi6[5], pi6[2]}};
    post_collision<double>(rho, u, p, omega, F, out);
}
void orc_moments(const double* f, double* rho, double* u, double* pi6) {
    double p[3][3];
    moments<double>(f, *rho, u, p);
    pi6[0] = p[0][0]; pi6[1] = p[1][1]; pi6[2] = p[2][2];
    pi6[3] = p[0][1]; pi6[4] = p[0][2]; pi6[5] = p[1][2];
}
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }
double orc_inflow_noise(uint64_t seed, int64_t x, int64_t y, int64_t t) { return inflow_noise(seed, x, y, t); }
double orc_inflow_noise_gauss(uint64_t seed, int64_t x, int64_t y, int64_t t) {
    return inflow_noise_gauss(seed, x, y, t);
}

// ---- real (FP64) simulation ------------------------------------------------
void* orc_create(const int64_t* dims, double tau, const double* F, const int* bc, const int64_t* inflow_i,
                 const double* inflow_d, uint64_t seed, int* status) {
    Sim<double>* s = new Sim<double>();
    Inflow in;
    std::memset(&in, 0, sizeof(in));
    if (inflow_i) {
        in.center2[0] = inflow_i[0]; in.center2[1] = inflow_i[1]; in.diameter = inflow_i[2];
        in.origin[0] = inflow_i[3]; in.origin[1] = inflow_i[4];
        in.noise_kind = (int)inflow_i[5];
    }
    if (inflow_d) { in.u_jet = inflow_d[0]; in.noise_amp = inflow_d[1]; }
    in.seed = seed;
    int st = validate_and_init(s, dims, tau, F, bc, &in);
    if (status) *status = st;
    if (st != 0) { delete s; return nullptr; }
    return s;
}
void orc_destroy(void* h) { delete static_cast<Sim<double>*>(h); }
// Forcing scheme: 0 = Luo term, 1 = Guo (R11; periodic and wall faces only).
int orc_set_forcing(void* h, int kind) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    if (kind != 0 && kind != 1) return -1;
    for (int f = 0; f < 6; ++f)
        if (kind == 1 && (s->bc[f] == BC_INFLOW || s->bc[f] == BC_OUTFLOW || s->bc[f] == BC_NEE_WALL)) return -1;
    s->forcing = kind;
    return 0;
}
// Sponge layer of width W (0: none) and strength K along the z+ end (R8).
int orc_set_sponge(void* h, int64_t width, double k) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    if (width < 0 || width >= s->n[2] || !(k >= 0.0)) return -1;
    s->sponge_w = width;
    s->sponge_k = k;
    return 0;
}
int orc_init_moments(void* h, const double* rho, const double* u, const double* pi) {
    init_from_moments(static_cast<Sim<double>*>(h), rho, u, pi);
    return 0;
}
int orc_set_force_field(void* h, const double* F3N) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    if (!F3N) { s->has_field = false; s->field.clear(); return 0; }
    s->field.assign(F3N, F3N + 3 * s->N());
    s->has_field = true;
    return 0;
}
int orc_step(void* h, int64_t nsteps) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    for (int64_t k = 0; k < nsteps; ++k) {
        step_once(*s);
        if (check_filled(*s) != 0) return -10;
    }
    return 0;
}
int orc_get_moments(void* h, double* rho, double* u, double* pi) {
    get_moments(static_cast<Sim<double>*>(h), rho, u, pi);
    return 0;
}
int orc_get_populations(void* h, double* f) {
    Sim<double>* s = static_cast<Sim<double>*>(h);
    std::memcpy(f, s->f.data(), sizeof(double) * s->f.size());
    return 0;
}
int64_t orc_time(void* h) { return static_cast<Sim<double>*>(h)->t; }
// OpenMP threads a parallel step uses (the team size of a parallel region).
int orc_threads() {
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
}

// ---- complex-step simulation (for derivative checks) ---------------------
// Runs nsteps from real initial moments with a complex per-node force field
// (Fre + i Fim, [3][N]) and returns the complex kinetic energy
// J = 1/2 sum_interior rho |u|^2 written with u.u (no conjugate) so that it
// stays holomorphic; Im J(F + i h v)/h is the directional derivative dJ/dF.v.
}  // extern "C"

namespace {
// nsteps of the complex simulation from real initial moments under the
// complex force field Fre + i Fim; returns a validate_and_init status.
int complex_sim_run(Sim<cplx>& s, const int64_t* dims, double tau, const int* bc, const double* rho,
                    const double* u, const double* pi, const double* Fre, const double* Fim, int64_t nsteps) {
    const double F0[3] = {0.0, 0.0, 0.0};
    int st = validate_and_init(&s, dims, tau, F0, bc, nullptr);
    if (st != 0) return st;
    const int64_t N = s.N();
    std::vector<cplx> r(N), uu(3 * N), p(6 * N);
    for (int64_t k = 0; k < N; ++k) r[k] = rho[k];
    for (int64_t k = 0; k < 3 * N; ++k) uu[k] = u[k];
    for (int64_t k = 0; k < 6 * N; ++k) p[k] = pi ? pi[k] : 0.0;
    init_from_moments(&s, r.data(), uu.data(), p.data());
    s.field.resize(3 * N);
    for (int64_t k = 0; k < 3 * N; ++k) s.field[k] = cplx(Fre ? Fre[k] : 0.0, Fim ? Fim[k] : 0.0);
    s.has_field = true;
    for (int64_t k = 0; k < nsteps; ++k) step_once(s);
    return 0;
}
}  // namespace

extern "C" {

int orc_complex_run(const int64_t* dims, double tau, const int* bc, const double* rho, const double* u,
                    const double* pi, const double* Fre, const double* Fim, int64_t nsteps, double* J_re,
                    double* J_im) {
    Sim<cplx> s;
    int st = complex_sim_run(s, dims, tau, bc, rho, u, pi, Fre, Fim, nsteps);
    if (st != 0) return st;
    cplx J = 0.0;
    for (int64_t z = s.lo(2); z <= s.hi(2); ++z)
        for (int64_t y = s.lo(1); y <= s.hi(1); ++y)
            for (int64_t x = s.lo(0); x <= s.hi(0); ++x) {
                cplx rr, v[3], pp[3][3];
                node_moments(s, s.idx(x, y, z), rr, v, pp);
                J += 0.5 * rr * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            }
    *J_re = J.real();
    *J_im = J.imag();
    return 0;
}

// The same run, returning the complex final moments (full lattice, the
// layout of orc_get_moments: rho [N], u [3][N], pi [6][N], real and imaginary
// parts in separate [10][N] arrays) so that any holomorphic objective of them
// can be differentiated by the complex step.
int orc_complex_run_moments(const int64_t* dims, double tau, const int* bc, const double* rho, const double* u,
                            const double* pi, const double* Fre, const double* Fim, int64_t nsteps, double* m_re,
                            double* m_im) {
    Sim<cplx> s;
    int st = complex_sim_run(s, dims, tau, bc, rho, u, pi, Fre, Fim, nsteps);
    if (st != 0) return st;
    const int64_t N = s.N();
    std::vector<cplx> r(N), uu(3 * N), p(6 * N);
    get_moments(&s, r.data(), uu.data(), p.data());
    for (int64_t k = 0; k < N; ++k) { m_re[k] = r[k].real(); m_im[k] = r[k].imag(); }
    for (int64_t k = 0; k < 3 * N; ++k) { m_re[N + k] = uu[k].real(); m_im[N + k] = uu[k].imag(); }
    for (int64_t k = 0; k < 6 * N; ++k) { m_re[4 * N + k] = p[k].real(); m_im[4 * N + k] = p[k].imag(); }
    return 0;
}

}  // extern "C"
