// FP64 CPU oracle for the two-dimensional (D2Q9) high-order thread-safe LB step.
//
// TEST INFRASTRUCTURE ONLY, like tslb_oracle.cpp: only the test-suite and the
// CPU-baseline leg of the benchmark load it; it shares no source with the
// CUDA library.
//
// What it computes (arXiv 2401.17074, Sec. 2, written for a D2Q9 lattice):
//   * D2Q9 with cs^2 = 1/3 and the weights of the tensor product D1Q3 x D1Q3;
//   * third-order Hermite equilibria (Eq. eqts) and third-order regularised
//     non-equilibrium populations from Pi^neq by the Hermite recursion
//     (Eq. noneqts), every tensor sum over the two axes (the xxx- and
//     yyy-type third-order Hermite polynomials vanish on D2Q9 by themselves);
//   * the thread-safe update f_i(x+c_i,t+1) = f^eq_i + (1-omega) f^neq_i plus
//     the Luo forcing term rho w_i c_i.F / cs^2 (Eq. pushLB, Sec. 3.1);
//   * moments rho, rho u, Pi^neq as sums over the populations (Sec. 2).
// The same readings as the three-dimensional oracle apply (R1-R6 there), with
// direction index i = (cx+1) + 3(cy+1) and opposite 8 - i.  Faces: periodic,
// or halfway bounce-back walls on the y faces (the y = 0 and y = ny-1 layers
// are solid; only interior nodes are updated and stored).
//
// Parity status: pinned by tests/test_oracle2d_pins.py (lattice isotropy,
// moment identities, rest state, conservation, forcing, Taylor-Green decay,
// Poiseuille convergence).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

const double CS2 = 1.0 / 3.0;
const double CS4 = CS2 * CS2;
const double CS6 = CS4 * CS2;

enum { BC2_PERIODIC = 0, BC2_BOUNCEBACK = 1 };

struct Lattice2 {
    int c[9][2];
    double w[9];
    Lattice2() {
        const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                const int i = (cx + 1) + 3 * (cy + 1);
                c[i][0] = cx;
                c[i][1] = cy;
                w[i] = w1[cx + 1] * w1[cy + 1];
            }
    }
    static int opp(int i) { return 8 - i; }
};
const Lattice2 L2;

inline double delta(int a, int b) { return a == b ? 1.0 : 0.0; }
inline double H2(const int* c, int a, int b) { return c[a] * c[b] - CS2 * delta(a, b); }
inline double H3(const int* c, int a, int b, int g) {
    return c[a] * c[b] * c[g] - CS2 * (c[g] * delta(a, b) + c[a] * delta(b, g) + c[b] * delta(a, g));
}

void feq3(double rho, const double u[2], double out[9]) {
    for (int i = 0; i < 9; ++i) {
        const int* c = L2.c[i];
        double cu = 0.0, s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < 2; ++a) cu += c[a] * u[a];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) s2 += H2(c, a, b) * u[a] * u[b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int g = 0; g < 2; ++g) s3 += H3(c, a, b, g) * u[a] * u[b] * u[g];
        out[i] = rho * L2.w[i] * (1.0 + cu / CS2 + s2 / (2.0 * CS4) + s3 / (6.0 * CS6));
    }
}

void fneq3(const double pi[2][2], const double u[2], double out[9]) {
    for (int i = 0; i < 9; ++i) {
        const int* c = L2.c[i];
        double s2 = 0.0, s3 = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) s2 += H2(c, a, b) * pi[a][b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int g = 0; g < 2; ++g) {
                    const double a3 = pi[a][b] * u[g] + u[a] * pi[b][g] + u[b] * pi[a][g];
                    s3 += H3(c, a, b, g) * a3;
                }
        out[i] = L2.w[i] * (s2 / (2.0 * CS4) + s3 / (6.0 * CS6));
    }
}

void moments(const double* f, double& rho, double u[2], double pi[2][2]) {
    rho = 0.0;
    double j[2] = {0.0, 0.0}, m2[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int i = 0; i < 9; ++i) {
        const int* c = L2.c[i];
        rho += f[i];
        for (int a = 0; a < 2; ++a) j[a] += c[a] * f[i];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) m2[a][b] += c[a] * c[b] * f[i];
    }
    for (int a = 0; a < 2; ++a) u[a] = j[a] / rho;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) pi[a][b] = m2[a][b] - rho * u[a] * u[b] - rho * CS2 * delta(a, b);
}

void post_collision(double rho, const double u[2], const double pi[2][2], double omega, const double F[2],
                    double out[9]) {
    double eq[9], neq[9];
    feq3(rho, u, eq);
    fneq3(pi, u, neq);
    for (int i = 0; i < 9; ++i) {
        const double cF = L2.c[i][0] * F[0] + L2.c[i][1] * F[1];
        out[i] = eq[i] + (1.0 - omega) * neq[i] + rho * L2.w[i] * cF / CS2;
    }
}

struct Sim2 {
    int64_t n[2];
    int bc[4];  // x-, x+, y-, y+
    double omega;
    double F[2];
    int64_t t;
    std::vector<double> f, fnew;  // [node][9]

    int64_t N() const { return n[0] * n[1]; }
    int64_t idx(int64_t x, int64_t y) const { return x + n[0] * y; }
    int64_t lo(int a) const { return bc[2 * a] == BC2_PERIODIC ? 0 : 1; }
    int64_t hi(int a) const { return bc[2 * a + 1] == BC2_PERIODIC ? n[a] - 1 : n[a] - 2; }
    bool interior(int64_t x, int64_t y) const { return x >= lo(0) && x <= hi(0) && y >= lo(1) && y <= hi(1); }
};

// One push-form step: every interior node emits its nine post-collision
// populations; a population that would enter a solid wall layer returns to
// its source as the opposite direction (halfway bounce-back).
void step_once(Sim2& s) {
    std::fill(s.fnew.begin(), s.fnew.end(), std::numeric_limits<double>::quiet_NaN());
#pragma omp parallel for schedule(static)
    for (int64_t y = s.lo(1); y <= s.hi(1); ++y)
        for (int64_t x = s.lo(0); x <= s.hi(0); ++x) {
            const int64_t node = s.idx(x, y);
            double rho, u[2], pi[2][2], post[9];
            moments(&s.f[node * 9], rho, u, pi);
            post_collision(rho, u, pi, s.omega, s.F, post);
            for (int i = 0; i < 9; ++i) {
                int64_t d[2] = {x + L2.c[i][0], y + L2.c[i][1]};
                bool bounce = false;
                for (int a = 0; a < 2; ++a) {
                    if (s.bc[2 * a] == BC2_PERIODIC) d[a] = (d[a] + s.n[a]) % s.n[a];
                    else if (d[a] < s.lo(a) || d[a] > s.hi(a)) bounce = true;
                }
                if (bounce) s.fnew[node * 9 + Lattice2::opp(i)] = post[i];
                else s.fnew[s.idx(d[0], d[1]) * 9 + i] = post[i];
            }
        }
    std::swap(s.f, s.fnew);
    s.t += 1;
}

int check_filled(const Sim2& s) {
    for (int64_t y = s.lo(1); y <= s.hi(1); ++y)
        for (int64_t x = s.lo(0); x <= s.hi(0); ++x)
            for (int i = 0; i < 9; ++i)
                if (std::isnan(s.f[s.idx(x, y) * 9 + i])) return -1;
    return 0;
}

}  // namespace

extern "C" {

void orc2_lattice(int* c /*9x2*/, double* w /*9*/) {
    for (int i = 0; i < 9; ++i) {
        c[2 * i] = L2.c[i][0];
        c[2 * i + 1] = L2.c[i][1];
        w[i] = L2.w[i];
    }
}
void orc2_feq3(double rho, const double* u, double* out) { feq3(rho, u, out); }
void orc2_fneq3(const double* pi3 /*xx, yy, xy*/, const double* u, double* out) {
    const double p[2][2] = {{pi3[0], pi3[2]}, {pi3[2], pi3[1]}};
    fneq3(p, u, out);
}
void orc2_moments(const double* f, double* rho, double* u, double* pi3) {
    double p[2][2];
    moments(f, *rho, u, p);
    pi3[0] = p[0][0];
    pi3[1] = p[1][1];
    pi3[2] = p[0][1];
}

// dims = (nx, ny); bc = (x-, x+, y-, y+) with 0 = periodic, 1 = bounce-back
// (y faces only); F = constant acceleration (2).  Returns NULL with *status < 0
// on a rejected configuration.
void* orc2_create(const int64_t* dims, double tau, const double* F, const int* bc, int* status) {
    int st = 0;
    if (!(tau > 0.5)) st = -2;
    for (int a = 0; a < 2 && st == 0; ++a) {
        if (bc[2 * a] != bc[2 * a + 1]) st = -3;
        else if (bc[2 * a] != BC2_PERIODIC && bc[2 * a] != BC2_BOUNCEBACK) st = -3;
        else if (a == 0 && bc[0] != BC2_PERIODIC) st = -3;
        else if (dims[a] < (bc[2 * a] == BC2_PERIODIC ? 3 : 4)) st = -4;
    }
    if (status) *status = st;
    if (st != 0) return nullptr;
    Sim2* s = new Sim2();
    for (int a = 0; a < 2; ++a) {
        s->n[a] = dims[a];
        s->bc[2 * a] = bc[2 * a];
        s->bc[2 * a + 1] = bc[2 * a + 1];
        s->F[a] = F ? F[a] : 0.0;
    }
    s->omega = 1.0 / tau;
    s->t = 0;
    s->f.assign(s->N() * 9, 0.0);
    s->fnew.assign(s->N() * 9, 0.0);
    return s;
}
void orc2_destroy(void* h) { delete static_cast<Sim2*>(h); }

// Full-lattice inputs: rho[N], u[2][N], pi[3][N] (xx, yy, xy; may be NULL).
// Populations start at f^eq3 + f^neq3 (the post-collision form with omega = 0).
int orc2_init_moments(void* h, const double* rho, const double* u, const double* pi) {
    Sim2* s = static_cast<Sim2*>(h);
    const int64_t N = s->N();
    for (int64_t y = s->lo(1); y <= s->hi(1); ++y)
        for (int64_t x = s->lo(0); x <= s->hi(0); ++x) {
            const int64_t node = s->idx(x, y);
            const double uu[2] = {u[node], u[N + node]};
            double p[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
            if (pi) {
                p[0][0] = pi[node];
                p[1][1] = pi[N + node];
                p[0][1] = p[1][0] = pi[2 * N + node];
            }
            double eq[9], neq[9];
            feq3(rho[node], uu, eq);
            fneq3(p, uu, neq);
            for (int i = 0; i < 9; ++i) s->f[node * 9 + i] = eq[i] + neq[i];
        }
    s->t = 0;
    return 0;
}
int orc2_step(void* h, int64_t nsteps) {
    Sim2* s = static_cast<Sim2*>(h);
    for (int64_t k = 0; k < nsteps; ++k) {
        step_once(*s);
        if (check_filled(*s) != 0) return -10;
    }
    return 0;
}
// Full-lattice outputs; solid layers report the rest state.
int orc2_get_moments(void* h, double* rho, double* u, double* pi) {
    Sim2* s = static_cast<Sim2*>(h);
    const int64_t N = s->N();
    for (int64_t y = 0; y < s->n[1]; ++y)
        for (int64_t x = 0; x < s->n[0]; ++x) {
            const int64_t node = s->idx(x, y);
            double r = 1.0, uu[2] = {0.0, 0.0}, p[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
            if (s->interior(x, y)) moments(&s->f[node * 9], r, uu, p);
            if (rho) rho[node] = r;
            if (u) {
                u[node] = uu[0];
                u[N + node] = uu[1];
            }
            if (pi) {
                pi[node] = p[0][0];
                pi[N + node] = p[1][1];
                pi[2 * N + node] = p[0][1];
            }
        }
    return 0;
}

}  // extern "C"
