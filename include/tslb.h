/*
 * tslb.h -- C ABI of the B300 (sm_103a) high-order thread-safe lattice
 * Boltzmann library (arXiv 2401.17074, "High-order thread-safe lattice
 * Boltzmann model for HPC turbulent flow simulations").
 *
 * The library advances a D3Q27 lattice whose state is only the 10 macroscopic
 * moment fields per node -- density rho, velocity u and the non-equilibrium
 * momentum flux Pi^neq (Sec. 2.1, the "10 arrays" of the thread-safe scheme).
 * One step rebuilds, at every node x, the post-collision populations of its
 * 26 neighbours x - c_i from their moments by third-order recursive Hermite
 * regularisation (Eq. eqts, Eq. noneqts, the combined update after
 * Eq. noneqts), streams them (Eq. pushLB, written in pull form) and sums the
 * new moments.  Body forcing (Luo term, Sec. 3.1) and wall / inflow / outflow
 * faces (Sec. 2.3, Sec. 3.2) are applied in the same pass.
 *
 * Conventions shared by every call:
 *   - Lattice coordinates (x, y, z) run over dims[0] x dims[1] x dims[2]
 *     nodes, x fastest; node index n = x + nx*(y + ny*z); N = nx*ny*nz.
 *   - A non-periodic face turns the outermost node layer on that side into a
 *     boundary layer: solid for BOUNCEBACK / FREESLIP (walls halfway between
 *     it and the first interior layer), a ghost layer for INFLOW / OUTFLOW.
 *     Only interior nodes are stored and updated; "interior nodes" below is
 *     the product of the interior extents.
 *   - Moment arrays exchanged with the caller are full-lattice FP64 arrays:
 *     rho[N]; u[3][N] (u_x, u_y, u_z planes); pi[6][N] in the order
 *     xx, yy, zz, xy, xz, yz.  Boundary-layer entries are ignored on input
 *     and returned as the rest state (rho = 1, u = 0, Pi = 0) on output.
 *   - `where` says whether a pointer is host memory (TSLB_HOST, pageable or
 *     pinned) or device memory on the handle's device (TSLB_DEVICE).  Device
 *     memory is read and written on the handle's stream only: work of other
 *     streams that produces an input, or still uses an output buffer, must be
 *     complete (or ordered before the handle's stream by an event) when the
 *     call is made.  The Python binding drains PyTorch's current stream
 *     before passing a CUDA tensor.
 *   - Every call returns TSLB_OK (0) or a negative tslb_status; on error the
 *     handle is unchanged unless stated and tslb_last_error() explains.  No
 *     call aborts the process or traps the device.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef TSLB_H
#define TSLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tslb_s tslb_t;

typedef enum tslb_status {
    TSLB_OK = 0,
    TSLB_ERR_INVALID = -1,     /* bad argument (null pointer, tau <= 1/2, size too small, ...) */
    TSLB_ERR_UNSUPPORTED = -2, /* valid request this library does not implement */
    TSLB_ERR_CUDA = -3,        /* a CUDA runtime call failed, or a kernel reported through the device
                                * status word: a bounded wait that gave up (the factored step's row
                                * exchange) or, in the index-checked build libtslb_checked.so, an
                                * index out of range; see tslb_last_error */
    TSLB_ERR_ALLOC = -4,       /* device or host allocation failed */
    TSLB_ERR_UNSTABLE = -5,    /* diagnostics found NaN/Inf in the moment fields */
    TSLB_ERR_STATE = -6        /* call not valid in the handle's current state */
} tslb_status;

/* Lattices.  TSLB_D2Q9 is the two-dimensional variant of the same step (the
 * recursion of Eq. noneqts on D1Q3 x D1Q3): dims = (nx, ny, 1) with periodic z
 * faces, periodic x, periodic or TSLB_BC_BOUNCEBACK y faces, FP32 storage, the
 * constant body force only (no force field, adjoint, inflow or sponge; the
 * `kernel` option is ignored).  Its moment arrays keep the three-dimensional
 * layouts: u_z, Pi_zz, Pi_xz and Pi_yz are ignored on input and returned as 0. */
enum { TSLB_D3Q27 = 27, TSLB_D2Q9 = 9 };

/* Face boundary conditions, indexed bc[0..5] = x-, x+, y-, y+, z-, z+. */
typedef enum tslb_bc {
    TSLB_BC_PERIODIC = 0,   /* both faces of the axis must be periodic */
    TSLB_BC_BOUNCEBACK = 1, /* halfway bounce-back no-slip wall (y faces only) */
    TSLB_BC_FREESLIP = 2,   /* halfway specular-reflection wall (x or y faces) */
    TSLB_BC_INFLOW = 3,     /* z- only: thread-safe Hermite non-equilibrium inflow, Eq. neq_final */
    TSLB_BC_OUTFLOW = 4,    /* z+ only: zero-gradient outflow (moments of the adjacent layer) */
    TSLB_BC_HALO = 6,       /* z faces only, both: this handle is one z slab of a larger lattice split along
                               z (the multi-GPU decomposition named as future work in the paper's
                               Conclusions).  Every node layer z = 0 .. nz-1 is interior; the step reads the
                               layers z = -1 and z = nz from two ghost planes, which the caller fills
                               between steps with the neighbouring slabs' boundary layers
                               (tslb_halo_export / tslb_halo_import).  D3Q27, factored kernel, periodic
                               x, periodic or bounce-back y, Luo forcing with the constant body force only
                               (no force field, sponge, checkpoints or adjoint) */
    TSLB_BC_NEE_WALL = 5    /* y faces only, with periodic x and z: no-slip wall on the boundary layer by
                               the thread-safe non-equilibrium extrapolation (Sec. 2.3, Eq. neq_final with
                               imposed momentum u_B = 0): each boundary node emits
                               f^eq(rho_F, 0) + (1 - omega) Hermite f^neq(Pi^neq, u of x_F), x_F the
                               adjacent interior node; the wall is on the node, so the channel half-width
                               is (ny - 1)/2 */
} tslb_bc;

typedef enum tslb_precision {
    TSLB_FP32 = 0, /* moments stored as FP32 (rho stored as rho - 1) */
    TSLB_BF16 = 1, /* stored as BF16 scaled deviations: rho-1, u/u_ref, Pi/pi_ref */
    TSLB_FP16 = 2  /* stored as FP16 scaled deviations */
} tslb_precision;

typedef enum tslb_where { TSLB_HOST = 0, TSLB_DEVICE = 1 } tslb_where;

/* Body-force schemes.  TSLB_FORCING_LUO is the paper's term rho w_i c_i.F/cs^2
 * added to the post-collision populations (Sec. 3.1).  TSLB_FORCING_GUO is Guo's
 * scheme: the stored velocity is u = (sum f c + rho F/2)/rho, the stored stress
 * is Pi = sum f c c - rho u u - rho cs^2 delta + (rho/2)(u F + F u), and the
 * post-collision populations are f^eq + (1 - omega) f^neq(Pi) + F_i/2 with
 * F_i = w_i rho [(c - u).F/cs^2 + (c.u)(c.F)/cs^4]; a uniformly accelerating
 * flow then carries no spurious stress.  Guo forcing needs TSLB_D3Q27 with
 * periodic x and z faces, y faces periodic, bounce-back or free-slip, no sponge
 * layer, and is not supported by tslb_adjoint_force_gradient. */
typedef enum tslb_forcing { TSLB_FORCING_LUO = 0, TSLB_FORCING_GUO = 1 } tslb_forcing;

/* Rounding of the 16-bit storage codecs when a step stores its moments.
 * TSLB_ROUND_NEAREST rounds every stored value to nearest even.
 * TSLB_ROUND_STOCHASTIC stores rho - 1 and u rounded up or down in magnitude with
 * probabilities that make the stored value exact in expectation (16 random bits
 * per value from a counter-based hash of (node, step, rounding_seed), so a run
 * is reproducible and both step kernels draw the same bits); Pi^neq keeps
 * rounding to nearest.  Rounding to nearest drops per-step increments below half
 * a 16-bit spacing (a body force of 1e-7 on u ~ 0.05 in BF16), so a forced flow
 * stops accelerating; stochastic rounding keeps them on average.  The initial
 * state is always rounded to nearest.  Requires TSLB_BF16 or TSLB_FP16. */
typedef enum tslb_rounding { TSLB_ROUND_NEAREST = 0, TSLB_ROUND_STOCHASTIC = 1 } tslb_rounding;

typedef enum tslb_kernel {
    TSLB_KERNEL_AUTO = 0,     /* the fastest kernel that supports the configuration */
    TSLB_KERNEL_DIRECT = 1,   /* one thread per node, 27 direct gathers (cross-check path) */
    TSLB_KERNEL_FACTORED = 2  /* sum-factorised, z-marching tiled kernel; up to 2^32 - 1 interior nodes
                                 (AUTO takes the direct kernel beyond) */
} tslb_kernel;

/* Inflow noise of the round jet (Sec. 3.2). */
typedef enum tslb_noise {
    TSLB_NOISE_UNIFORM = 0, /* xi uniform in [-1, 1): (r0 >> 8) 2^-23 - 1 */
    TSLB_NOISE_GAUSSIAN = 1 /* xi ~ N(0, 1), the paper's "time-varying Gaussian noise": Box-Muller,
                               xi = sqrt(-2 ln u1) cos(2 pi u2), u1 = ((r0 >> 8) + 1) 2^-24,
                               u2 = (r1 >> 8) 2^-24 */
} tslb_noise;

/* Inflow nozzle of the round jet (Sec. 3.2): inside the disc
 * (2x - center2[0])^2 + (2y - center2[1])^2 <= diameter^2 the imposed velocity
 * is u_z = u_jet (1 + noise_amp * xi), with xi drawn per column (x, y) and per
 * step t from the Philox4x32-10 block of counter (x, y, t, 0) and key `seed`
 * (r0, r1 its first two words) as `noise_kind` says; outside it is zero. */
typedef struct tslb_inflow {
    int64_t center2[2];
    int64_t diameter;
    double u_jet;
    double noise_amp;
    uint64_t seed;
    int noise_kind;       /* tslb_noise, default TSLB_NOISE_UNIFORM */
} tslb_inflow;

typedef struct tslb_options {
    int precision;        /* tslb_precision, default TSLB_FP32 */
    double u_ref;         /* velocity scale of 16-bit storage, default 0.05 */
    double pi_ref;        /* Pi^neq scale of 16-bit storage, default 1e-3 */
    void* stream;         /* cudaStream_t to run on; NULL = a stream owned by the handle */
    int device;           /* CUDA device ordinal, default 0 */
    int kernel;           /* tslb_kernel, default TSLB_KERNEL_AUTO */
    int checkpoint_every; /* >0: tslb_step records a moment checkpoint every k steps (adjoint); the
                           * checkpoint buffers are reused by later runs until tslb_destroy */
    tslb_inflow inflow;   /* used when bc[4] == TSLB_BC_INFLOW */
    /* Sponge layer towards the z+ face (the jet's exit, Sec. 3.2): with
     * W = sponge_width > 0 (default 0 = none) and z_s = nz - W, a node at
     * lattice z > z_s relaxes with nu(z) = nu (1 + sponge_k ((z - z_s)/W)^3),
     * nu = cs^2 (tau - 1/2), i.e. omega(z) = 1 / (1/2 + nu(z)/cs^2).  The
     * paper prints the exponent as -3 (which diverges at z_s) and normalises by
     * an undefined z_end; +3 and W are this library's reading.  Requires
     * W < nz and sponge_k >= 0; not supported by tslb_adjoint_force_gradient. */
    int sponge_width;
    double sponge_k;
    int forcing;          /* tslb_forcing, default TSLB_FORCING_LUO */
    int rounding;         /* tslb_rounding, default TSLB_ROUND_NEAREST */
    uint64_t rounding_seed; /* key of the stochastic rounding bits, default 0 */
    /* Halo slabs only: cudaStream_t on which tslb_halo_export / tslb_halo_import
     * run (NULL = the handle's stream, default).  With a separate stream the
     * library orders the copies against the steps with events, so an exchange
     * can overlap a split step's interior part (tslb_step_part). */
    void* halo_stream;
} tslb_options;

typedef struct tslb_diag {
    double mass;           /* sum over interior nodes of rho */
    double momentum[3];    /* sum of rho u */
    double kinetic_energy; /* 1/2 sum rho |u|^2 */
    double wall_shear;     /* y walls: mean of -(1-omega/2) Pi_xy on y=1 and +(...) on y=ny-2; else 0 */
    double max_speed;      /* max |u| (Mach check) */
    int64_t nonfinite;     /* number of interior nodes with a NaN/Inf moment */
    int64_t steps;         /* steps taken since tslb_init_moments */
    int64_t nodes;         /* interior nodes */
} tslb_diag;

/* Fill *opt with the defaults listed above.  Returns TSLB_ERR_INVALID if opt is NULL. */
int tslb_options_default(tslb_options* opt);

/* Create a solver (problem statement of Sec. 2 and Sec. 3: lattice, grid, tau
 * with nu = cs^2 (tau - 1/2), constant body-force acceleration `force`
 * (Sec. 3.1; NULL = 0), face conditions `bc`).  The library allocates and owns
 * all device memory (two buffers of the 10 moment fields).  Rejects tau <= 1/2,
 * an axis shorter than 3 (periodic) or 4 (otherwise), mixed periodic /
 * non-periodic faces on one axis (TSLB_ERR_INVALID), and any lattice other than
 * TSLB_D3Q27 or a face combination not listed in tslb_bc (TSLB_ERR_UNSUPPORTED).
 * *out is written only on success.  The moment fields start at the rest state. */
int tslb_create(tslb_t** out, int lattice, const int64_t dims[3], double tau, const double force[3],
                const int bc[6], const tslb_options* opt);

/* Load the moment fields (Sec. 2.1: rho, u, Pi^neq) from full-lattice FP64
 * arrays; `pi` may be NULL (Pi^neq = 0).  The caller keeps ownership; the call
 * returns after the data are copied.  Resets the step counter to 0. */
int tslb_init_moments(tslb_t* h, const double* rho, const double* u, const double* pi, int where);

/* The same with FP32 arrays and the density given as its deviation drho = rho - 1
 * (the stored quantity, so that FP32 keeps its precision): drho [N], u [3][N],
 * pi [6][N] (may be NULL), full lattice, host or device per `where`.  With FP32
 * storage a moment read back by tslb_get_moments_f32 is bit-identical to the
 * value loaded.  Half the bytes of the FP64 form cross the host link.
 * TSLB_D3Q27 only (TSLB_ERR_UNSUPPORTED otherwise). */
int tslb_init_moments_f32(tslb_t* h, const float* drho, const float* u, const float* pi, int where);

/* Per-node body-force acceleration F[3][N] (FP32, full lattice) replacing the
 * constant force; NULL restores the constant force given to tslb_create. */
int tslb_set_force_field(tslb_t* h, const float* F, int where);

/* Advance nsteps TSLB steps (Eq. pushLB with Eq. eqts / Eq. noneqts
 * reconstruction, forcing and faces), asynchronously on the handle's stream.
 * Launch errors are reported immediately; the call does not synchronise.
 * Each step is one kernel launched with programmatic stream serialisation:
 * its set-up may overlap the end of the kernel before it on the stream, but
 * it reads and writes global memory only after that kernel has completed, so
 * stream order holds for any work the caller puts on the same stream. */
int tslb_step(tslb_t* h, int64_t nsteps);

/* Copy the current moments out as full-lattice FP64 arrays (any pointer may
 * be NULL to skip that field).  Synchronises the handle's stream. */
int tslb_get_moments(tslb_t* h, double* rho, double* u, double* pi, int where);

/* The same into FP32 arrays, with the density as drho = rho - 1 (see
 * tslb_init_moments_f32).  TSLB_D3Q27 only. */
int tslb_get_moments_f32(tslb_t* h, float* drho, float* u, float* pi, int where);

/* FP64 reductions over the interior nodes (mass, momentum, kinetic energy,
 * wall shear, max |u|, NaN/Inf count).  Synchronises the stream.  Returns
 * TSLB_ERR_UNSTABLE (with *out filled) if any moment is NaN or Inf. */
int tslb_diagnostics(tslb_t* h, tslb_diag* out);

/* Gradient of J = 1/2 sum rho |u|^2 at the current step with respect to a
 * time-constant per-node body-force field, back-propagated through the last
 * `nsteps` steps taken since tslb_init_moments by the discrete adjoint of the
 * step.  Requires options.checkpoint_every > 0 at create time; segments
 * between checkpoints are recomputed.  dJdF is a full-lattice FP32 [3][N]
 * array (boundary entries 0).  Synchronises the stream.  The first call
 * allocates a workspace of checkpoint_every moment states plus 23 FP32 values
 * per node, which the handle keeps for later calls until tslb_destroy.
 * Boxes of fewer than 2^31 nodes with periodic faces, or periodic x and z
 * with halfway bounce-back walls on the y faces (the channel); Luo forcing, no
 * sponge layer; TSLB_ERR_UNSUPPORTED otherwise. */
int tslb_adjoint_force_gradient(tslb_t* h, int64_t nsteps, float* dJdF, int where);

/* Gradient dJ/dF of any objective J of the final moments with respect to the
 * time-constant per-node body-force field (Luo term of Sec. 3.1), through the
 * last `nsteps` steps -- the discrete adjoint of the step of Sec. 2.1-2.2
 * (Eq. eqts, Eq. noneqts, Eq. pushLB), run backwards from the caller's seed.
 * lambda_T is the cotangent dJ/dm of the current (final) moments as a
 * full-lattice FP64 [10][N] array: rows rho (equally rho - 1), u_x, u_y, u_z,
 * Pi_xx, Pi_yy, Pi_zz, Pi_xy, Pi_xz, Pi_yz, each the derivative with respect
 * to the stored component (Pi_xy counted once); boundary-layer entries are
 * ignored.  The caller keeps ownership; it is read before the call returns.
 * ckpt_every is 0 or the checkpoint_every the handle was created with
 * (TSLB_ERR_INVALID otherwise).  dJdF is a full-lattice FP32 [3][N] array
 * (boundary entries 0).  `where` applies to lambda_T and dJdF.  A host
 * lambda_T is staged through 80 bytes per lattice node of device memory that
 * the handle allocates on first use and keeps until tslb_destroy.  Otherwise
 * as tslb_adjoint_force_gradient, which is the special case
 * lambda = (|u|^2/2, rho u, 0) of J = 1/2 sum rho |u|^2.  Synchronises the
 * stream. */
int tslb_adjoint(tslb_t* h, const double* lambda_T, int64_t nsteps, int ckpt_every, float* dJdF, int where);

/* ---- Diagnostics without allocation ------------------------------------
 * The paper has no counterpart of this call.  It serves callers that cannot
 * allocate device memory at the point where they want the numbers: programs
 * run under a fixed device-memory budget that is already spent, programs whose
 * framework allocator has reserved all of the device's memory up front (a
 * plain cudaMalloc then fails although the framework holds free blocks), and
 * latency-bound loops between solver steps, where cudaMalloc / cudaFree, which
 * may synchronise the whole device, are not acceptable.
 *
 * tslb_diagnostics_noalloc computes the same FP64 sums as tslb_diagnostics
 * over moment arrays the caller owns: rho[N], u[3][N] and pi[6][N] (pi may be
 * NULL) in the full-lattice FP64 layout that tslb_get_moments(..., TSLB_DEVICE)
 * writes, in device memory of the current device.  dims and bc describe the
 * lattice as for tslb_create (only interior nodes are summed); tau sets the
 * wall-shear factor (1 - 1/(2 tau)).  It launches two kernels on `stream`
 * (NULL = the default stream) and returns without synchronising; `out` (device
 * memory, 8 doubles) then holds mass, momentum x, y, z, kinetic energy, wall
 * shear, max |u| and the number of interior nodes with a NaN/Inf value.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine: the per-block
 * partial sums live in a fixed 256 KB __device__ array that every device
 * loading this library holds until the process exits.  Consequences:
 *   - at most TSLB_NOALLOC_MAX_NODES interior nodes; more return TSLB_ERR_INVALID;
 *   - the first call on a device does the set-up: it looks up the array's
 *     device address with cudaGetSymbolAddress, with that device current, and
 *     keeps it for the life of the process; make that first call before any
 *     stream capture.  The address belongs to the device's primary context:
 *     after cudaDeviceReset of that device, do not call this entry point again
 *     in the same process;
 *   - a node counts as non-finite when any of its moments (rho, u and, when
 *     pi is given, the six Pi components) is NaN or Inf;
 *   - every call shares the array: calls that overlap on the GPU (other
 *     streams, other host threads) race and give wrong sums.  Each call
 *     rewrites every partial it reads, so nothing carries over between calls.
 * Errors return a negative tslb_status; tslb_last_error(NULL) explains. */
#define TSLB_NOALLOC_MAX_NODES ((int64_t)1 << 26)
int tslb_diagnostics_noalloc(const double* rho, const double* u, const double* pi, const int64_t dims[3],
                             const int bc[6], double tau, void* stream, double* out);

/* ---- Slab decomposition along z (TSLB_BC_HALO faces) --------------------
 * The paper's Conclusions name the multi-GPU extension as future work; its
 * natural form for the thread-safe step is a split of the lattice into z
 * slabs, one handle per slab, whose steps need one layer of the 10 stored
 * moment fields from each neighbour per time step.  A packed plane holds the
 * nx * ny interior nodes of one layer as the three stored arrays in turn
 * (V0 = (u_x, u_y, u_z, rho - 1), V1 = (Pi_xx, Pi_yy, Pi_zz, Pi_xy),
 * V2 = (Pi_xz, Pi_yz)), in the handle's storage type: 10 * nx * ny values.
 * One exchange per step, before it: for each slab s,
 *   tslb_halo_export(s, 1, buf)  ->  tslb_halo_import(next slab, 0, buf)
 *   tslb_halo_export(s, 0, buf)  ->  tslb_halo_import(previous slab, 1, buf)
 * with the slabs in a ring (z periodic overall).  Both calls run on the
 * handle's stream (device buffers) or complete before returning (host
 * buffers); a device buffer shared by two handles on different streams must
 * be ordered between them by the caller (an event, or one shared stream).
 * With options.halo_stream set, both run on that stream and the library
 * orders them against the steps with events: an export waits for the layers
 * it reads (the last step, or an open step's edges), an import for the last
 * step or open step's edges that read the ghosts it overwrites, and the next
 * step (or EDGES part) waits for the imports.  The caller then orders its
 * buffers with respect to that stream only.
 * These calls return TSLB_ERR_STATE on a handle without TSLB_BC_HALO faces. */

/* Bytes of one packed plane. */
int tslb_halo_plane_bytes(const tslb_t* h, int64_t* bytes);

/* A step of a halo slab in two parts, so that the exchange of its boundary
 * layers can overlap the update of the rest:
 *   TSLB_PART_EDGES    advances the layers z < e and z >= nz - e
 *                      (e = TSLB_HALO_EDGE_LAYERS, or all layers when nz <= 2e);
 *   TSLB_PART_INTERIOR advances the layers in between and completes the step.
 * Between the two the step is open: tslb_halo_export exports the layers z = 0
 * and z = nz - 1 of the state being produced (already final), and
 * tslb_halo_import loads the ghosts of the next step (the open step's edges
 * no longer read them).  EDGES then INTERIOR equals one tslb_step bit for bit.
 * TSLB_ERR_STATE for EDGES while a step is open, INTERIOR while none is, or
 * tslb_step while one is; TSLB_ERR_STATE on a handle without halo faces. */
enum { TSLB_PART_EDGES = 1, TSLB_PART_INTERIOR = 2 };
#define TSLB_HALO_EDGE_LAYERS 4
int tslb_step_part(tslb_t* h, int part);

/* Copy this slab's boundary layer -- side 0: z = 0, side 1: z = nz - 1, at the
 * current step -- into dst as one packed plane (host or device per `where`). */
int tslb_halo_export(tslb_t* h, int side, void* dst, int where);

/* Load a packed plane into the ghost plane the next step reads -- side 0: the
 * layer below z = 0 (the previous slab's z = nz - 1), side 1: the layer above
 * z = nz - 1 (the next slab's z = 0).  The ghost planes start at the rest
 * state and keep their contents until the next import. */
int tslb_halo_import(tslb_t* h, int side, const void* src, int where);

/* Number of interior (updated) nodes. */
int64_t tslb_interior_nodes(const tslb_t* h);

/* Block until all work queued on the handle's stream is done, then report the
 * device status word (TSLB_ERR_CUDA if a kernel recorded a failure since the
 * last report; the word is cleared). */
int tslb_synchronize(tslb_t* h);

/* Release all memory of the handle.  NULL is ignored. */
void tslb_destroy(tslb_t* h);

/* Text of the last error on this handle (never NULL).  For h == NULL, the
 * last error of a failed tslb_create on this thread. */
const char* tslb_last_error(const tslb_t* h);

#ifdef __cplusplus
}
#endif

#endif /* TSLB_H */
