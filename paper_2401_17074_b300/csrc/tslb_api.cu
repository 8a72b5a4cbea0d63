// C ABI of the TSLB library (declared in include/tslb.h): argument checks,
// device memory ownership, stream handling and kernel dispatch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tslb_internal.cuh"
#include <nvtx3/nvToolsExt.h>

namespace {

// NVTX range around a host call (visible in Nsight Systems / ncu range filters;
// a no-op unless a tool is attached).  For the asynchronous calls it covers the
// host side: argument checks and the launches.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

}  // namespace

namespace {

thread_local std::string g_create_error;

int fail(tslb_s* h, int code, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(tslb_s* h, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, TSLB_ERR_CUDA, m);
}

// Host-side fault injection for the error-path tests: TSLB_FAULT=alloc makes
// every device allocation of the library report failure without calling CUDA.
bool inject_alloc_fault() {
    const char* f = std::getenv("TSLB_FAULT");
    return f && std::strcmp(f, "alloc") == 0;
}

// TSLB_FAULT=exchange makes one warp row of the factored step withhold its
// y-exchange arrival, so that its neighbours' bounded waits run out (about a
// second) and the step reports the device status word.
bool inject_exchange_fault() {
    const char* f = std::getenv("TSLB_FAULT");
    return f && std::strcmp(f, "exchange") == 0;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_alloc_async(void** p, size_t bytes, cudaStream_t s) {
    if (inject_alloc_fault()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, s);
}

bool valid_handle(const tslb_s* h) { return h != nullptr; }

// After a synchronise: report a bounded device wait that gave up (bit 2; the
// kernel then skipped the rest of its work) or, in the checked build, an index
// out of range (bit 4; the access was skipped), and clear the word.
int check_device_status(tslb_s* h) {
    int v = 0;
    if (!h->dev_err) return TSLB_OK;
    cudaError_t e = cudaMemcpy(&v, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (v != 0) {
        cudaMemset(h->dev_err, 0, sizeof(int));
        std::string m;
        if (v & 2) m += "a bounded device wait gave up; ";
        if (v & TSLB_ERR_BIT_INDEX) m += "an index check of the checked build failed; ";
        return fail(h, TSLB_ERR_CUDA, m + "the step results are invalid");
    }
    return TSLB_OK;
}

void release(tslb_s* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (int b = 0; b < 2; ++b)
        if (h->buf[b]) cudaFree(h->buf[b]);
    if (h->force_field) cudaFree(h->force_field);
    if (h->diag_part) cudaFree(h->diag_part);
    if (h->dev_err) cudaFree(h->dev_err);
    if (h->omega1_z) cudaFree(h->omega1_z);
    if (h->diag_host) cudaFreeHost(h->diag_host);
    for (void* c : h->ckpts) cudaFree(c);
    if (h->adj_ws) cudaFree(h->adj_ws);
    if (h->adj_lam) cudaFree(h->adj_lam);
    if (h->ghost) cudaFree(h->ghost);
    if (h->ev_step) cudaEventDestroy(h->ev_step);
    if (h->ev_edges) cudaEventDestroy(h->ev_edges);
    if (h->ev_halo) cudaEventDestroy(h->ev_halo);
    if (h->halo_stream && h->halo_stream != h->stream) cudaStreamSynchronize(h->halo_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // namespace

namespace tslb {

void set_global_error(const std::string& msg) { g_create_error = msg; }

Physics make_physics(const tslb_s* h) {
    Physics p{};
    p.omega1 = (float)(1.0 - h->omega);
    for (int a = 0; a < 3; ++a) p.F[a] = (float)h->force[a];
    p.force = h->force_field;
    p.in_c2[0] = h->inflow.center2[0];
    p.in_c2[1] = h->inflow.center2[1];
    p.in_d = h->inflow.diameter;
    p.in_u = (float)h->inflow.u_jet;
    p.in_amp = (float)h->inflow.noise_amp;
    p.in_seed = h->inflow.seed;
    p.in_gauss = h->inflow.noise_kind == TSLB_NOISE_GAUSSIAN ? 1 : 0;
    p.omega1_z = h->omega1_z;
    p.guo = h->forcing == TSLB_FORCING_GUO ? 1 : 0;
    p.t = h->t;
    p.err = h->dev_err;
    p.drop_row = inject_exchange_fault() ? 5 : -1;
    if (h->precision == TSLB_FP32) {
        p.s_u = p.s_pi = p.inv_s_u = p.inv_s_pi = 1.0f;
    } else {
        p.s_u = (float)h->u_ref;
        p.s_pi = (float)h->pi_ref;
        p.inv_s_u = (float)(1.0 / h->u_ref);
        p.inv_s_pi = (float)(1.0 / h->pi_ref);
    }
    p.sr_key = sr_step_key(h->rounding_seed, h->t);
    if (h->ghost) {
        p.halo[0] = h->ghost;
        p.halo[1] = static_cast<const char*>(h->ghost) + halo_ghost_stride(h);
    }
    p.omega1_pi = (float)((1.0 - h->omega) * (double)p.s_pi);
    p.pi_store = (float)((double)p.inv_s_pi / 216.0);
    return p;
}

bool use_factored(const tslb_s* h) { return h->kernel != TSLB_KERNEL_DIRECT && factored_supports(h); }

cudaError_t launch_step_any(const tslb_s* h, const void* src, void* dst, const Physics& p) {
    if (h->lattice == TSLB_D2Q9) return launch_step2d(h, src, dst, p);
    return use_factored(h) ? launch_step_factored(h, src, dst, p) : launch_step_direct(h, src, dst, p);
}

}  // namespace tslb

namespace {

size_t state_bytes(const tslb_s* h) { return (size_t)h->nfields * h->g.fstride * h->elem; }

// Forget the recorded checkpoints; their buffers are reused by the next run
// (copies into them are ordered on the handle's stream).
void drop_checkpoints(tslb_s* h) { h->ckpt_valid = 0; }

}  // namespace

namespace tslb {
cudaError_t launch_encode_f32(const tslb_s* h, const float* drho, const float* u, const float* pi, void* dst,
                              const Physics& p);
cudaError_t launch_decode_f32(const tslb_s* h, const void* src, float* drho, float* u, float* pi, const Physics& p);
}  // namespace tslb

namespace {

// Host element type of the moment arrays: FP64 rho, or FP32 rho - 1.
cudaError_t encode_any(const tslb_s* h, const double* r, const double* u, const double* pi, void* dst,
                       const tslb::Physics& p) {
    return tslb::launch_encode(h, r, u, pi, dst, p);
}
cudaError_t encode_any(const tslb_s* h, const float* r, const float* u, const float* pi, void* dst,
                       const tslb::Physics& p) {
    return tslb::launch_encode_f32(h, r, u, pi, dst, p);
}
cudaError_t decode_any(const tslb_s* h, const void* src, double* r, double* u, double* pi, const tslb::Physics& p) {
    return tslb::launch_decode(h, src, r, u, pi, p);
}
cudaError_t decode_any(const tslb_s* h, const void* src, float* r, float* u, float* pi, const tslb::Physics& p) {
    return tslb::launch_decode_f32(h, src, r, u, pi, p);
}

template <class H>
int init_moments_impl(tslb_t* h, const H* rho, const H* u, const H* pi, int where) {
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (!rho || !u) return fail(h, TSLB_ERR_INVALID, "rho (or drho) and u are required");
    if (where != TSLB_HOST && where != TSLB_DEVICE) return fail(h, TSLB_ERR_INVALID, "bad 'where'");
    if (h->step_open) return fail(h, TSLB_ERR_STATE, "a split step is open");
    cudaSetDevice(h->device);
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    const tslb::Physics p = tslb::make_physics(h);
    cudaError_t e;
    if (where == TSLB_DEVICE) {
        e = encode_any(h, rho, u, pi, h->buf[h->cur], p);
        if (e != cudaSuccess) return cuda_fail(h, e, "encode launch");
    } else {
        H* st = nullptr;
        const size_t bytes = sizeof(H) * (size_t)fN * (pi ? 10 : 4);
        e = dev_alloc_async((void**)&st, bytes, h->stream);
        if (e != cudaSuccess) return fail(h, TSLB_ERR_ALLOC, "staging allocation failed");
        e = cudaMemcpyAsync(st, rho, sizeof(H) * fN, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st + fN, u, sizeof(H) * 3 * fN, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess && pi)
            e = cudaMemcpyAsync(st + 4 * fN, pi, sizeof(H) * 6 * fN, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = encode_any(h, st, st + fN, pi ? st + 4 * fN : nullptr, h->buf[h->cur], p);
        cudaFreeAsync(st, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "init copy / encode");
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "init synchronize");
    h->t = 0;
    drop_checkpoints(h);
    return TSLB_OK;
}

template <class H>
int get_moments_impl(tslb_t* h, H* rho, H* u, H* pi, int where) {
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (where != TSLB_HOST && where != TSLB_DEVICE) return fail(h, TSLB_ERR_INVALID, "bad 'where'");
    cudaSetDevice(h->device);
    const long long fN = h->dims[0] * h->dims[1] * h->dims[2];
    const tslb::Physics p = tslb::make_physics(h);
    cudaError_t e;
    if (where == TSLB_DEVICE) {
        e = decode_any(h, h->buf[h->cur], rho, u, pi, p);
        if (e != cudaSuccess) return cuda_fail(h, e, "decode launch");
    } else {
        H* st = nullptr;
        e = dev_alloc_async((void**)&st, sizeof(H) * (size_t)fN * 10, h->stream);
        if (e != cudaSuccess) return fail(h, TSLB_ERR_ALLOC, "staging allocation failed");
        e = decode_any(h, h->buf[h->cur], rho ? st : nullptr, u ? st + fN : nullptr,
                                pi ? st + 4 * fN : nullptr, p);
        if (e == cudaSuccess && rho)
            e = cudaMemcpyAsync(rho, st, sizeof(H) * fN, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && u)
            e = cudaMemcpyAsync(u, st + fN, sizeof(H) * 3 * fN, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && pi)
            e = cudaMemcpyAsync(pi, st + 4 * fN, sizeof(H) * 6 * fN, cudaMemcpyDeviceToHost, h->stream);
        cudaFreeAsync(st, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "get copy / decode");
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "get synchronize");
    return check_device_status(h);
}

}  // namespace

extern "C" {

int tslb_options_default(tslb_options* opt) {
    if (!opt) return TSLB_ERR_INVALID;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = TSLB_FP32;
    opt->u_ref = 0.05;
    opt->pi_ref = 1e-3;
    opt->stream = nullptr;
    opt->device = 0;
    opt->kernel = TSLB_KERNEL_AUTO;
    opt->checkpoint_every = 0;
    opt->halo_stream = nullptr;
    return TSLB_OK;
}

int tslb_create(tslb_t** out, int lattice, const int64_t dims[3], double tau, const double force[3],
                const int bc[6], const tslb_options* opt) {
    const Range range("tslb_create");
    g_create_error.clear();
    if (!out || !dims || !bc) return fail(nullptr, TSLB_ERR_INVALID, "null argument");
    if (lattice != TSLB_D3Q27 && lattice != TSLB_D2Q9)
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "lattices: TSLB_D3Q27 or TSLB_D2Q9");
    const bool d2 = lattice == TSLB_D2Q9;
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(nullptr, TSLB_ERR_INVALID, "tau must be > 1/2");
    for (int f = 0; f < 6; ++f)
        if (bc[f] < TSLB_BC_PERIODIC || bc[f] > TSLB_BC_HALO)
            return fail(nullptr, TSLB_ERR_INVALID, "unknown boundary code");
    for (int a = 0; a < 3; ++a) {
        const bool p0 = bc[2 * a] == TSLB_BC_PERIODIC, p1 = bc[2 * a + 1] == TSLB_BC_PERIODIC;
        if (p0 != p1) return fail(nullptr, TSLB_ERR_INVALID, "an axis mixes periodic and non-periodic faces");
        if (d2 && a == 2) {
            if (dims[2] != 1 || !p0) return fail(nullptr, TSLB_ERR_INVALID, "D2Q9 needs nz = 1 with periodic z faces");
            continue;
        }
        // a halo slab has no boundary layer: every layer is interior, as on a periodic axis
        const bool halo = bc[2 * a] == TSLB_BC_HALO;
        if (dims[a] < (p0 || halo ? 3 : 4)) return fail(nullptr, TSLB_ERR_INVALID, "axis too short");
        if (dims[a] > (int64_t)1 << 30) return fail(nullptr, TSLB_ERR_INVALID, "axis too long");
    }
    // Supported face combinations (see tslb_bc).
    const int bx = bc[0], by = bc[2], bz0 = bc[4], bz1 = bc[5];
    if (bc[0] != bc[1] || bc[2] != bc[3])
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "x and y faces must match pairwise");
    if (!(bx == TSLB_BC_PERIODIC || bx == TSLB_BC_FREESLIP))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "x faces: periodic or free-slip");
    if (!(by == TSLB_BC_PERIODIC || by == TSLB_BC_FREESLIP || by == TSLB_BC_BOUNCEBACK || by == TSLB_BC_NEE_WALL))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "y faces: periodic, bounce-back, free-slip or NEE wall");
    for (int f = 0; f < 4; ++f)
        if (bc[f] == TSLB_BC_HALO) return fail(nullptr, TSLB_ERR_UNSUPPORTED, "halo faces are z faces");
    const bool zhalo = bz0 == TSLB_BC_HALO && bz1 == TSLB_BC_HALO;
    if (!((bz0 == TSLB_BC_PERIODIC && bz1 == TSLB_BC_PERIODIC) || (bz0 == TSLB_BC_INFLOW && bz1 == TSLB_BC_OUTFLOW) ||
          zhalo))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "z faces: periodic, inflow (z-) with outflow (z+), or both halo");
    // a halo slab's z layers are interior like a periodic axis's, for every face rule below
    const bool zper_like = bz0 == TSLB_BC_PERIODIC || zhalo;
    if ((by == TSLB_BC_BOUNCEBACK || by == TSLB_BC_NEE_WALL) && (bx != TSLB_BC_PERIODIC || !zper_like))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "bounce-back and NEE y walls need periodic x and z");

    tslb_options o;
    if (opt) o = *opt;
    else tslb_options_default(&o);
    if (o.precision < TSLB_FP32 || o.precision > TSLB_FP16)
        return fail(nullptr, TSLB_ERR_INVALID, "unknown precision");
    if (o.precision != TSLB_FP32 && (!(o.u_ref > 0) || !(o.pi_ref > 0)))
        return fail(nullptr, TSLB_ERR_INVALID, "16-bit storage needs positive u_ref and pi_ref");
    if (o.kernel < TSLB_KERNEL_AUTO || o.kernel > TSLB_KERNEL_FACTORED)
        return fail(nullptr, TSLB_ERR_INVALID, "unknown kernel choice");
    if (o.checkpoint_every < 0) return fail(nullptr, TSLB_ERR_INVALID, "checkpoint_every < 0");
    if (bz0 == TSLB_BC_INFLOW && o.inflow.diameter < 0) return fail(nullptr, TSLB_ERR_INVALID, "bad inflow diameter");
    if (d2 && (bx != TSLB_BC_PERIODIC || !(by == TSLB_BC_PERIODIC || by == TSLB_BC_BOUNCEBACK)))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "D2Q9: periodic x, periodic or bounce-back y");
    if (o.forcing != TSLB_FORCING_LUO && o.forcing != TSLB_FORCING_GUO)
        return fail(nullptr, TSLB_ERR_INVALID, "unknown forcing scheme");
    if (o.rounding != TSLB_ROUND_NEAREST && o.rounding != TSLB_ROUND_STOCHASTIC)
        return fail(nullptr, TSLB_ERR_INVALID, "unknown rounding mode");
    if (o.rounding == TSLB_ROUND_STOCHASTIC && o.precision == TSLB_FP32)
        return fail(nullptr, TSLB_ERR_INVALID, "stochastic rounding applies to 16-bit storage");
    if (zhalo && (d2 || o.kernel == TSLB_KERNEL_DIRECT || o.sponge_width != 0 || o.checkpoint_every != 0 ||
                  bx != TSLB_BC_PERIODIC || !(by == TSLB_BC_PERIODIC || by == TSLB_BC_BOUNCEBACK) ||
                  o.forcing != TSLB_FORCING_LUO))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED,
                    "halo slabs: D3Q27, factored kernel, periodic x, periodic or bounce-back y, Luo forcing, "
                    "no sponge layer, no checkpoints");
    if (o.forcing == TSLB_FORCING_GUO &&
        (d2 || bx != TSLB_BC_PERIODIC || !zper_like || by == TSLB_BC_NEE_WALL || o.sponge_width != 0))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED,
                    "Guo forcing: D3Q27, periodic x and z, no NEE walls, no sponge layer");
    if (d2 && (o.precision != TSLB_FP32 || o.checkpoint_every != 0 || o.sponge_width != 0))
        return fail(nullptr, TSLB_ERR_UNSUPPORTED, "D2Q9: FP32 storage, no checkpoints, no sponge layer");
    if (o.inflow.noise_kind != TSLB_NOISE_UNIFORM && o.inflow.noise_kind != TSLB_NOISE_GAUSSIAN)
        return fail(nullptr, TSLB_ERR_INVALID, "unknown inflow noise kind");
    if (o.sponge_width < 0 || o.sponge_width >= dims[2] || !(o.sponge_k >= 0.0) || !std::isfinite(o.sponge_k))
        return fail(nullptr, TSLB_ERR_INVALID, "sponge layer needs 0 <= width < nz and K >= 0");

    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (o.device < 0 || o.device >= ndev) return fail(nullptr, TSLB_ERR_INVALID, "bad device ordinal");

    tslb_s* h = new tslb_s();
    h->device = o.device;
    h->lattice = lattice;
    h->nfields = d2 ? 6 : (int)tslb::NFIELDS;
    for (int a = 0; a < 3; ++a) h->dims[a] = dims[a];
    for (int f = 0; f < 6; ++f) h->bc[f] = bc[f];
    h->tau = tau;
    h->omega = 1.0 / tau;
    for (int a = 0; a < 3; ++a) h->force[a] = force ? force[a] : 0.0;
    h->precision = o.precision;
    h->u_ref = o.u_ref;
    h->pi_ref = o.pi_ref;
    h->kernel = o.kernel;
    h->checkpoint_every = o.checkpoint_every;
    h->inflow = o.inflow;
    h->sponge_width = o.sponge_width;
    h->forcing = o.forcing;
    h->rounding = o.rounding;
    h->rounding_seed = o.rounding_seed;
    h->sponge_k = o.sponge_k;
    h->elem = o.precision == TSLB_FP32 ? 4 : 2;

    tslb::Geometry& g = h->g;
    int ext[3];
    for (int a = 0; a < 3; ++a) {
        const bool per = bc[2 * a] == TSLB_BC_PERIODIC || bc[2 * a] == TSLB_BC_HALO;
        g.lo[a] = per ? 0 : 1;
        ext[a] = (int)(per ? dims[a] : dims[a] - 2);
    }
    g.nx = ext[0];
    g.ny = ext[1];
    g.nz = ext[2];
    for (int f = 0; f < 6; ++f) g.bc[f] = bc[f];
    g.plane = (long long)g.nx * g.ny;
    const long long Ni = g.plane * g.nz;
    g.fstride = (Ni + 127) / 128 * 128;  // 512-byte aligned field planes (FP32)

    e = cudaSetDevice(h->device);
    if (e != cudaSuccess) {
        int r = cuda_fail(nullptr, e, "cudaSetDevice");
        delete h;
        return r;
    }
    if (o.stream) {
        h->stream = (cudaStream_t)o.stream;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            int r = cuda_fail(nullptr, e, "cudaStreamCreate");
            delete h;
            return r;
        }
        h->own_stream = true;
    }
    const size_t bytes = (size_t)h->nfields * g.fstride * h->elem;
    for (int b = 0; b < 2; ++b) {
        e = dev_alloc(&h->buf[b], bytes);
        if (e != cudaSuccess) {
            std::string m = std::string("device allocation of the moment fields failed: ") + cudaGetErrorString(e);
            release(h);
            return fail(nullptr, TSLB_ERR_ALLOC, m);
        }
        e = cudaMemsetAsync(h->buf[b], 0, bytes, h->stream);  // zero deviations = rest state
        if (e != cudaSuccess) {
            release(h);
            return cuda_fail(nullptr, e, "cudaMemsetAsync");
        }
    }
    if (h->sponge_width > 0) {
        // (1 - omega) per full-lattice z: nu(z) = nu (1 + K ((z - z_s)/W)^3) above z_s = nz - W
        const int64_t nzf = dims[2], W = h->sponge_width, zs = nzf - W;
        const double nu0 = (tau - 0.5) / 3.0;
        std::vector<float> tab((size_t)nzf);
        for (int64_t z = 0; z < nzf; ++z) {
            double nu = nu0;
            if (z > zs) {
                const double r = (double)(z - zs) / (double)W;
                nu = nu0 * (1.0 + h->sponge_k * r * r * r);
            }
            tab[(size_t)z] = (float)(1.0 - 1.0 / (0.5 + 3.0 * nu));
        }
        e = dev_alloc((void**)&h->omega1_z, sizeof(float) * (size_t)nzf);
        if (e != cudaSuccess) {
            std::string m = std::string("device allocation of the sponge table failed: ") + cudaGetErrorString(e);
            release(h);
            return fail(nullptr, TSLB_ERR_ALLOC, m);
        }
        e = cudaMemcpy(h->omega1_z, tab.data(), sizeof(float) * (size_t)nzf, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            release(h);
            return cuda_fail(nullptr, e, "sponge table copy");
        }
    }
    if (zhalo) {
        // the two ghost planes the step reads at z = -1 and z = nz (packed, rest state)
        const size_t gb = 2 * halo_ghost_stride(h);
        e = dev_alloc(&h->ghost, gb);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ghost, 0, gb, h->stream);
        h->halo_stream = o.halo_stream ? (cudaStream_t)o.halo_stream : h->stream;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_step, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_edges, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_halo, cudaEventDisableTiming);
        // the ghosts' rest state is written on the handle's stream: imports on
        // another stream come after it
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_step, h->stream);
        if (e != cudaSuccess) {
            std::string m = std::string("device allocation of the ghost planes failed: ") + cudaGetErrorString(e);
            release(h);
            return fail(nullptr, TSLB_ERR_ALLOC, m);
        }
    }
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    h->sm_count = sms;
    h->diag_blocks = sms * 4;
    e = dev_alloc((void**)&h->diag_part, sizeof(double) * 8 * (h->diag_blocks + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&h->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->diag_host, sizeof(double) * 8);
    if (e != cudaSuccess) {
        std::string m = std::string("device allocation of the diagnostics scratch failed: ") + cudaGetErrorString(e);
        release(h);
        return fail(nullptr, TSLB_ERR_ALLOC, m);
    }
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        release(h);
        return cuda_fail(nullptr, e, "cudaStreamSynchronize");
    }
    *out = h;
    return TSLB_OK;
}

int tslb_init_moments(tslb_t* h, const double* rho, const double* u, const double* pi, int where) {
    const Range range("tslb_init_moments");
    return init_moments_impl<double>(h, rho, u, pi, where);
}

int tslb_init_moments_f32(tslb_t* h, const float* drho, const float* u, const float* pi, int where) {
    const Range range("tslb_init_moments_f32");
    if (valid_handle(h) && h->lattice != TSLB_D3Q27)
        return fail(h, TSLB_ERR_UNSUPPORTED, "FP32 host moments are implemented for D3Q27");
    return init_moments_impl<float>(h, drho, u, pi, where);
}

int tslb_set_force_field(tslb_t* h, const float* F, int where) {
    const Range range("tslb_set_force_field");
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (where != TSLB_HOST && where != TSLB_DEVICE) return fail(h, TSLB_ERR_INVALID, "bad 'where'");
    if (h->lattice == TSLB_D2Q9) return fail(h, TSLB_ERR_UNSUPPORTED, "D2Q9 takes the constant body force only");
    if (h->ghost && F) return fail(h, TSLB_ERR_UNSUPPORTED, "halo slabs take the constant body force only");
    cudaSetDevice(h->device);
    if (!F) {
        if (h->force_field) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->force_field);
        }
        h->force_field = nullptr;
        return TSLB_OK;
    }
    const tslb::Geometry& g = h->g;
    cudaError_t e;
    if (!h->force_field) {
        e = dev_alloc((void**)&h->force_field, sizeof(float) * 4 * g.fstride);
        if (e != cudaSuccess) {
            h->force_field = nullptr;
            return fail(h, TSLB_ERR_ALLOC, "force field allocation failed");
        }
    }
    // Gather the interior of the full-lattice [3][N] array row by row into a
    // planar staging array, then interleave it into one float4 per node.
    float* planar = nullptr;
    e = dev_alloc_async((void**)&planar, sizeof(float) * 3 * g.fstride, h->stream);
    if (e != cudaSuccess) return fail(h, TSLB_ERR_ALLOC, "force field staging allocation failed");
    const long long fnx = h->dims[0], fny = h->dims[1], fN = fnx * fny * h->dims[2];
    const cudaMemcpyKind kind = where == TSLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        const float* srcA = F + a * fN;
        float* dstA = planar + a * g.fstride;
        for (int z = 0; z < g.nz; ++z) {
            const float* s = srcA + g.lo[0] + fnx * (g.lo[1] + fny * (long long)(z + g.lo[2]));
            e = cudaMemcpy2DAsync(dstA + g.plane * z, sizeof(float) * g.nx, s, sizeof(float) * fnx,
                                  sizeof(float) * g.nx, g.ny, kind, h->stream);
            if (e != cudaSuccess) break;
        }
    }
    if (e == cudaSuccess) e = tslb::launch_pack_force(h, planar, h->force_field);
    cudaFreeAsync(planar, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "force field copy");
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "force field synchronize");
    return TSLB_OK;
}

int tslb_step(tslb_t* h, int64_t nsteps) {
    const Range range("tslb_step");
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (nsteps < 0) return fail(h, TSLB_ERR_INVALID, "nsteps < 0");
    if (h->step_open) return fail(h, TSLB_ERR_STATE, "a split step is open: call tslb_step_part(TSLB_PART_INTERIOR)");
    cudaSetDevice(h->device);
    if (h->lattice == TSLB_D3Q27 && (h->kernel == TSLB_KERNEL_FACTORED || h->ghost) && !tslb::factored_supports(h))
        return fail(h, TSLB_ERR_UNSUPPORTED, "the factored kernel does not support this configuration");
    const int k = h->checkpoint_every;
    for (int64_t s = 0; s < nsteps; ++s) {
        cudaError_t e;
        if (k > 0 && h->t % k == 0 && h->ckpt_valid == h->t / k) {
            if ((size_t)h->ckpt_valid == h->ckpts.size()) {
                void* c = nullptr;
                e = dev_alloc(&c, state_bytes(h));
                if (e != cudaSuccess) return fail(h, TSLB_ERR_ALLOC, "checkpoint allocation failed");
                h->ckpts.push_back(c);
            }
            void* c = h->ckpts[(size_t)h->ckpt_valid];
            e = cudaMemcpyAsync(c, h->buf[h->cur], state_bytes(h), cudaMemcpyDeviceToDevice, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "checkpoint copy");
            ++h->ckpt_valid;
        }
        const tslb::Physics p = tslb::make_physics(h);
        const bool sep = h->ghost && h->halo_stream != h->stream;
        if (sep) cudaStreamWaitEvent(h->stream, h->ev_halo, 0);  // the ghosts this step reads
        e = tslb::launch_step_any(h, h->buf[h->cur], h->buf[h->cur ^ 1], p);
        if (e == cudaSuccess && sep) e = cudaEventRecord(h->ev_step, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
        h->cur ^= 1;
        h->t += 1;
    }
    return TSLB_OK;
}

int tslb_step_part(tslb_t* h, int part) {
    const Range range("tslb_step_part");
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (part != TSLB_PART_EDGES && part != TSLB_PART_INTERIOR) return fail(h, TSLB_ERR_INVALID, "unknown part");
    if (!h->ghost) return fail(h, TSLB_ERR_STATE, "split steps are for halo slabs");
    if (part == TSLB_PART_EDGES && h->step_open) return fail(h, TSLB_ERR_STATE, "a split step is already open");
    if (part == TSLB_PART_INTERIOR && !h->step_open) return fail(h, TSLB_ERR_STATE, "no split step is open");
    if (!tslb::factored_supports(h)) return fail(h, TSLB_ERR_UNSUPPORTED, "lattice too large for the factored kernel");
    cudaSetDevice(h->device);
    const tslb::Physics p = tslb::make_physics(h);
    const int nz = h->g.nz, ed = TSLB_HALO_EDGE_LAYERS;
    const bool whole = nz <= 2 * ed;  // the edges are the whole slab
    const bool sep = h->halo_stream != h->stream;
    cudaError_t e = cudaSuccess;
    void* src = h->buf[h->cur];
    void* dst = h->buf[h->cur ^ 1];
    if (part == TSLB_PART_EDGES) {
        if (sep) e = cudaStreamWaitEvent(h->stream, h->ev_halo, 0);
        if (e == cudaSuccess) e = tslb::launch_step_factored_range(h, src, dst, p, 0, whole ? nz : ed);
        if (e == cudaSuccess && !whole) e = tslb::launch_step_factored_range(h, src, dst, p, nz - ed, nz);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_edges, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step launch (edges)");
        h->step_open = true;
        return TSLB_OK;
    }
    if (!whole) e = tslb::launch_step_factored_range(h, src, dst, p, ed, nz - ed);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_step, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch (interior)");
    h->step_open = false;
    h->cur ^= 1;
    h->t += 1;
    return TSLB_OK;
}

int tslb_get_moments(tslb_t* h, double* rho, double* u, double* pi, int where) {
    const Range range("tslb_get_moments");
    return get_moments_impl<double>(h, rho, u, pi, where);
}

int tslb_get_moments_f32(tslb_t* h, float* drho, float* u, float* pi, int where) {
    const Range range("tslb_get_moments_f32");
    if (valid_handle(h) && h->lattice != TSLB_D3Q27)
        return fail(h, TSLB_ERR_UNSUPPORTED, "FP32 host moments are implemented for D3Q27");
    return get_moments_impl<float>(h, drho, u, pi, where);
}

int tslb_diagnostics(tslb_t* h, tslb_diag* out) {
    const Range range("tslb_diagnostics");
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (!out) return fail(h, TSLB_ERR_INVALID, "null output");
    cudaSetDevice(h->device);
    const tslb::Physics p = tslb::make_physics(h);
    double* dev_out = h->diag_part + 8 * h->diag_blocks;
    cudaError_t e = tslb::launch_diag(h, h->buf[h->cur], p, dev_out);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->diag_host, dev_out, sizeof(double) * 8, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "diagnostics");
    const int st = check_device_status(h);
    if (st != TSLB_OK) return st;
    const double* d = h->diag_host;
    out->mass = d[0];
    out->momentum[0] = d[1];
    out->momentum[1] = d[2];
    out->momentum[2] = d[3];
    out->kinetic_energy = d[4];
    const bool ywalls = h->bc[2] == TSLB_BC_BOUNCEBACK || h->bc[2] == TSLB_BC_NEE_WALL;
    out->wall_shear = ywalls ? d[5] / (2.0 * (double)h->g.nx * (double)h->g.nz) : 0.0;
    out->max_speed = d[6];
    out->nonfinite = (int64_t)d[7];
    out->steps = h->t;
    out->nodes = (int64_t)h->g.plane * h->g.nz;
    if (out->nonfinite > 0) return fail(h, TSLB_ERR_UNSTABLE, "NaN or Inf in the moment fields");
    return TSLB_OK;
}

// Checks shared by the two adjoint entry points, then the sweep.
static int adjoint_common(tslb_t* h, const double* lambda, int64_t nsteps, float* dJdF, int where) {
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (!dJdF) return fail(h, TSLB_ERR_INVALID, "null output");
    if (where != TSLB_HOST && where != TSLB_DEVICE) return fail(h, TSLB_ERR_INVALID, "bad 'where'");
    if (h->omega1_z) return fail(h, TSLB_ERR_UNSUPPORTED, "the adjoint does not support a sponge layer");
    if (h->lattice == TSLB_D2Q9) return fail(h, TSLB_ERR_UNSUPPORTED, "the adjoint is implemented for D3Q27");
    if (h->forcing != TSLB_FORCING_LUO) return fail(h, TSLB_ERR_UNSUPPORTED, "the adjoint is implemented for Luo forcing");
    cudaSetDevice(h->device);
    std::string msg;
    const int r = tslb::adjoint_run(h, lambda, nsteps, dJdF, where, &msg);
    if (r != TSLB_OK) return fail(h, r, msg);
    return TSLB_OK;
}

int tslb_adjoint_force_gradient(tslb_t* h, int64_t nsteps, float* dJdF, int where) {
    const Range range("tslb_adjoint_force_gradient");
    return adjoint_common(h, nullptr, nsteps, dJdF, where);
}

int tslb_adjoint(tslb_t* h, const double* lambda_T, int64_t nsteps, int ckpt_every, float* dJdF, int where) {
    const Range range("tslb_adjoint");
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (!lambda_T) return fail(h, TSLB_ERR_INVALID, "null cotangent");
    if (ckpt_every != 0 && ckpt_every != h->checkpoint_every)
        return fail(h, TSLB_ERR_INVALID, "ckpt_every must be 0 or the handle's checkpoint_every");
    return adjoint_common(h, lambda_T, nsteps, dJdF, where);
}

int tslb_halo_plane_bytes(const tslb_t* h, int64_t* bytes) {
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (!bytes) return fail(const_cast<tslb_t*>(h), TSLB_ERR_INVALID, "null output");
    if (!h->ghost) return fail(const_cast<tslb_t*>(h), TSLB_ERR_STATE, "the handle has no halo faces");
    *bytes = (int64_t)halo_plane_bytes(h);
    return TSLB_OK;
}

// One packed plane <-> the three stored arrays of layer z (V0: 4 values per
// node, V1: 4, V2: 2, each array fs nodes apart), on the handle's stream.
static int halo_copy(tslb_t* h, int side, void* other, int where, bool to_other) {
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    if (!other) return fail(h, TSLB_ERR_INVALID, "null buffer");
    if (side != 0 && side != 1) return fail(h, TSLB_ERR_INVALID, "side must be 0 or 1");
    if (where != TSLB_HOST && where != TSLB_DEVICE) return fail(h, TSLB_ERR_INVALID, "bad 'where'");
    if (!h->ghost) return fail(h, TSLB_ERR_STATE, "the handle has no halo faces");
    cudaSetDevice(h->device);
    const tslb::Geometry& g = h->g;
    const size_t pb = halo_plane_bytes(h), e4 = 4 * h->elem * (size_t)g.plane, e2 = 2 * h->elem * (size_t)g.plane;
    cudaStream_t hs = h->halo_stream;
    const bool sep = hs != h->stream;
    // on a separate stream: after the layers an export reads, or the ghost
    // reads an import overwrites (the last step, or an open step's edges)
    cudaError_t e = sep ? cudaStreamWaitEvent(hs, h->step_open ? h->ev_edges : h->ev_step, 0) : cudaSuccess;
    if (e == cudaSuccess && to_other) {
        // layer z = 0 or nz - 1 of the newest state -> packed [V0 | V1 | V2]
        const char* b = static_cast<const char*>(h->buf[h->step_open ? h->cur ^ 1 : h->cur]);
        const size_t z = side == 0 ? 0 : (size_t)g.nz - 1, fsb = (size_t)g.fstride * h->elem;
        const cudaMemcpyKind kind = where == TSLB_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        char* d = static_cast<char*>(other);
        e = cudaMemcpyAsync(d, b + z * e4, e4, kind, hs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + e4, b + 4 * fsb + z * e4, e4, kind, hs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d + 2 * e4, b + 8 * fsb + z * e2, e2, kind, hs);
    } else if (e == cudaSuccess) {
        const cudaMemcpyKind kind = where == TSLB_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        e = cudaMemcpyAsync(static_cast<char*>(h->ghost) + side * halo_ghost_stride(h), other, pb, kind, hs);
        if (e == cudaSuccess && sep) e = cudaEventRecord(h->ev_halo, hs);
    }
    if (e == cudaSuccess && where == TSLB_HOST) e = cudaStreamSynchronize(hs);
    if (e != cudaSuccess) return cuda_fail(h, e, to_other ? "halo export" : "halo import");
    return TSLB_OK;
}

int tslb_halo_export(tslb_t* h, int side, void* dst, int where) {
    const Range range("tslb_halo_export");
    return halo_copy(h, side, dst, where, true);
}

int tslb_halo_import(tslb_t* h, int side, const void* src, int where) {
    const Range range("tslb_halo_import");
    return halo_copy(h, side, const_cast<void*>(src), where, false);
}

int64_t tslb_interior_nodes(const tslb_t* h) { return h ? (int64_t)h->g.plane * h->g.nz : 0; }

int tslb_synchronize(tslb_t* h) {
    if (!valid_handle(h)) return fail(nullptr, TSLB_ERR_INVALID, "null handle");
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "synchronize");
    return check_device_status(h);
}

void tslb_destroy(tslb_t* h) { release(h); }

const char* tslb_last_error(const tslb_t* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
