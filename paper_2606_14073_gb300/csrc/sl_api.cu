// sl_api.cu -- C ABI of the NEP-SPIN spin-lattice library (declared in include/spinlat.h).
//
// create_system / step / energy_forces_fields follow the problem statement of
// arXiv 2606.14073 (Section 5.2.1: one unified energy E(R,S) giving forces and
// spin driving terms, advanced by the spin-lattice integrator).  All arrays
// crossing the ABI are host arrays in caller atom order; internally atoms are
// stored species-major and in Morton order of 7 A cells for locality.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/spinlat.h"
#include "sl_internal.h"
#include "sl_batch.h"

// NVTX range over a host-side call (shows up in profilers that record NVTX; a no-op otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct sl_system {
    sl::Sys s;
};

// Replicas stepped together, in a fixed number of slots (null: empty).  When the replicas
// taking part in a call share the device and the model and none uses the midpoint iteration,
// they take the fused step (sl_batch.h): one launch of each kernel covers all of them, from
// captured graphs over device tables that outlive admissions and retirements.  Otherwise,
// when every occupied slot takes at least steps_per_graph steps, one captured graph holding
// every replica's steps (each on its own stream, forked from and joined to the batch stream)
// advances them together; else each replica's own graphs are queued on its stream.
struct sl_batch {
    std::vector<sl_system *> sys;     // slots
    cudaStream_t stream = nullptr;
    cudaGraphExec_t graph = nullptr;  // the fork/join graph
    int graph_steps = 0;
    std::vector<uint64_t> graph_uids;     // unique ids of the slots' systems when it was built (0: empty)
    std::vector<uint64_t> versions;   // and their capture versions
    std::vector<cudaEvent_t> ev;      // fork/join events: [0] batch, [1 + i] slot i
    int64_t graph_launches = 0;
    int64_t fused_steps = 0, kernel_launches = 0, fused_calls = 0, replica_calls = 0;
    int64_t reserve_atoms = 0;        // atoms the fused launches are sized for (sl_batch_reserve)
    // a submitted call not yet waited for: the slots taking part and their step counts
    std::vector<std::pair<int, int64_t>> in_flight;
    sl::FusedBatch fused;
    ~sl_batch() {
        if (graph) cudaGraphExecDestroy(graph);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
    } while (0)

template <typename T>
int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SL_ENOMEM, "cudaMalloc of %zu bytes failed: %s", sizeof(T) * count, cudaGetErrorString(e));
    }
    return SL_OK;
}

uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    auto spread = [](uint64_t v) {
        v &= 0x1fffff;
        v = (v | v << 32) & 0x1f00000000ffffULL;
        v = (v | v << 16) & 0x1f0000ff0000ffULL;
        v = (v | v << 8) & 0x100f00f00f00f00fULL;
        v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
        v = (v | v << 2) & 0x1249249249249249ULL;
        return v;
    };
    return spread(x) | spread(y) << 1 | spread(z) << 2;
}

template <typename R>
void fill_params(sl::NepDev<R> &P, const sl_nep_params *p) {
    using namespace sl;
    for (int a = 0; a < NS; ++a)
        for (int b = 0; b < NS; ++b)
            for (int g = 0; g < 6; ++g)
                for (int n = 0; n < NCH; ++n)
                    for (int k = 0; k < NK; ++k)
                        P.c[a][b][g][n][k] = (R)p->coeffs[((((a * NS) + b) * 6 + g) * NCH + n) * NK + k];
    for (int v = 0; v < DIM; ++v) P.scal[v] = (R)p->q_scaler[v];
    for (int h = 0; h < NH; ++h) {
        for (int v = 0; v < DIM; ++v) P.w0[h][v] = (R)p->w0[h * DIM + v];
        P.b0[h] = (R)p->b0[h];
        P.w1[h] = (R)p->w1[h];
    }
    P.b1 = (R)p->b1;
    P.rc_r = (R)p->rc_rad;
    P.rc_a = (R)p->rc_ang;
    P.inv_rc_r = (R)(1.0 / p->rc_rad);
    P.inv_rc_a = (R)(1.0 / p->rc_ang);
    P.rc_r2 = (R)(p->rc_rad * p->rc_rad);
    P.rc_a2 = (R)(p->rc_ang * p->rc_ang);
}

void free_sys(sl::Sys &s) {
    void *ptrs[] = {s.pos, s.vel, s.spin, s.spin_prev, s.F, s.H, s.posref, s.posf, s.spinf, s.species, s.orig,
                    s.inv, s.nbr, s.rev, s.nbr_hash, s.cells.posf, s.cells.key, s.seg, s.cells.count, s.cells.start, s.cells.fill, s.cells.atoms,
                    s.cells.of, s.cells.sub, s.q, s.bsum, s.fp, s.ei, s.pairs, s.clj, s.cls, s.cnt, s.cmask, s.fown, s.gii,
                    s.wpart, s.Fo, s.Ho,
                    s.status, s.rebuild, s.d_step, s.d_par, s.red, s.snap, s.d_builds,
                    s.posmid, s.posmidf, s.mids, s.midsf, s.mx, s.mg, s.aax, s.aag, s.aapart, s.md, s.Bat,
                    s.tex_acc, s.tex_m, s.tex_part, s.colour, s.mlp_img};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    sl::solo_free(s);
    if (s.h_par) cudaFreeHost(s.h_par);
    if (s.h_stage) cudaFreeHost(s.h_stage);
    if (s.h_status) cudaFreeHost(s.h_status);
    if (s.h_red) cudaFreeHost(s.h_red);
    if (s.graph) cudaGraphExecDestroy(s.graph);
    if (s.own_stream && s.stream) cudaStreamDestroy(s.stream);
}

void compute_step_params(const sl::Sys &s, double dt, double T, const double B[3], sl::StepDev &P) {
    using namespace sl;
    P.dt = dt;
    P.half_dt = 0.5 * dt;
    P.c_fric = std::exp(-s.gamma * dt);
    for (int t = 0; t < NS; ++t) {
        P.acc_m[t] = ACC / s.mass[t];
        P.sig_v[t] = T > 0 ? std::sqrt((1.0 - P.c_fric * P.c_fric) * KB * T * ACC / s.mass[t]) : 0.0;
        for (int c = 0; c < 3; ++c) P.zee[t][c] = s.moment[t] * MUB * B[c];
        P.mom[t] = s.moment[t] * MUB;
    }
    P.sig_eta = (T > 0 && s.lambda > 0 && dt > 0) ? std::sqrt(2.0 * s.lambda * KB * T * HBAR / dt) : 0.0;
    P.lambda = s.lambda;
    P.wscale = 1.0 / ((1.0 + s.lambda * s.lambda) * HBAR);
    P.disp2 = 0.25 * s.skin * s.skin;
    P.sts = s.sts;
    P.lng = s.lng;
    P.lng_drift = 0.0;
    P.lng_sig = 0.0;
    for (int t = 0; t < NS; ++t) P.landau[t][0] = P.landau[t][1] = 0.0;
    if (s.lng) {   // precession about H/hbar; damping and noise enter through the longitudinal terms
        P.sig_eta = 0.0;
        P.lambda = 0.0;
        P.wscale = 1.0 / HBAR;
        P.lng_drift = s.lng_alpha * dt / HBAR;
        P.lng_sig = (T > 0 && s.lng_alpha > 0) ? std::sqrt(2.0 * s.lng_alpha * KB * T * dt / HBAR) : 0.0;
        for (int t = 0; t < NS; ++t) { P.landau[t][0] = s.landau[t][0]; P.landau[t][1] = s.landau[t][1]; }
    }
}

int upload_params(sl::Sys &s, double dt, double T, const double B[3]) {
    // the pinned host block may still be read by an earlier copy in flight
    CK(cudaStreamSynchronize(s.stream));
    compute_step_params(s, dt, T, B, *s.h_par);
    s.last_dt = dt;
    s.last_T = T;
    CK(cudaMemcpyAsync(s.d_par, s.h_par, sizeof(sl::StepDev), cudaMemcpyHostToDevice, s.stream));
    return SL_OK;
}

void enqueue_step(sl::Sys &s) {
    sl::launch_first_half(s);
    sl::launch_rebuild(s, true);
    if (s.mid_iters > 0) {          // self-consistent midpoint spin update, then the end state
        sl::launch_midpoint(s);
        sl::launch_eval(s, false);
        sl::launch_second_half_nospin(s);
    } else {
        sl::launch_eval(s, false);
        sl::launch_second_half(s);
    }
}

int64_t kernels_per_step(const sl::Sys &s) { return sl::KERNELS_PER_STEP + sl::midpoint_kernels_per_step(s); }

// Evaluate at the current state: optional unconditional rebuild, eval, gather.
int evaluate(sl::Sys &s, bool rebuild, bool carried, bool want_virial) {
    if (s.n == 0) return SL_OK;
    if (rebuild) {
        sl::launch_rebuild(s, false);
        s.n_builds++;
    }
    sl::launch_eval(s, want_virial);
    sl::launch_gather(s, carried);
    CK(cudaGetLastError());
    return SL_OK;
}

int check_status(sl::Sys &s) {
    CK(cudaMemcpyAsync(s.h_status, s.status, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    const int st = *s.h_status;
    if (st & sl::ST_NBR_OVERFLOW)
        return fail(SL_ENBR_OVERFLOW, "neighbour list capacity exceeded (caps %d/%d)", s.cap, s.cap_ang);
    if (st & sl::ST_NONFINITE) return fail(SL_ENONFINITE, "non-finite force or field");
    if (st & sl::ST_TIMEOUT) return fail(SL_ETIMEOUT, "a bounded device wait gave up (tensor-core network)");
    if (st & sl::ST_MID_RANGE)
        return fail(SL_ENBR_OVERFLOW, "midpoint configuration moved beyond skin/2 of the list positions");
    return SL_OK;
}

// Pinned staging buffer of n records for state transfers (allocated once per system).
static double4 *stage_buffer(const sl::Sys &s) {
    if (!s.h_stage && cudaMallocHost((void **)&s.h_stage, sizeof(double4) * (size_t)s.n) != cudaSuccess) {
        s.h_stage = nullptr;
        return nullptr;
    }
    return s.h_stage;
}

// fn(lo, hi) over [0, n) in contiguous chunks on up to 8 host threads (one thread for small n);
// every index is handled by exactly one thread, so results do not depend on the split.
template <typename F>
static void parallel_chunks(int64_t n, F fn) {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t nt = n < 65536 ? 1 : std::min<int64_t>(std::min<unsigned>(hw, 8u), n / 32768);
    if (nt <= 1) {
        fn((int64_t)0, n);
        return;
    }
    // a thread that cannot be created (std::system_error, or bad_alloc for its vector slot)
    // leaves its chunk, and every later one, to the calling thread: no exception crosses the ABI
    std::vector<std::thread> th;
    int64_t started = 1;   // chunks [1, started) run on their own threads
    try {
        th.reserve((size_t)nt - 1);
        for (; started < nt; ++started) th.emplace_back(fn, n * started / nt, n * (started + 1) / nt);
    } catch (...) {
    }
    fn((int64_t)0, n / nt);
    for (int64_t t = started; t < nt; ++t) fn(n * t / nt, n * (t + 1) / nt);
    for (auto &x : th) x.join();
}

// host (caller order) -> device (internal order), through the pinned staging buffer
int upload_vec(sl::Sys &s, double4 *dst, const double *src, bool normalise) {
    double4 *h = stage_buffer(s);
    if (!h) return fail(SL_ENOMEM, "pinned staging buffer allocation failed");
    // the buffer may still be read by an earlier copy on this stream
    CK(cudaStreamSynchronize(s.stream));
    const int32_t *orig = s.h_orig.data();
    std::atomic<int> zero{0};
    parallel_chunks(s.n, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            const double *p = src + 3 * (int64_t)orig[i];
            double x = p[0], y = p[1], z = p[2];
            if (normalise) {
                // spins that are unit to rounding are kept bit for bit (exact resume)
                const double n2 = x * x + y * y + z * z;
                if (!(n2 > 0)) {
                    zero.store(1);
                    continue;
                }
                if (std::fabs(n2 - 1.0) > 1e-13) {
                    const double nn = std::sqrt(n2);
                    x /= nn; y /= nn; z /= nn;
                }
            }
            h[i] = make_double4(x, y, z, 0.0);
        }
    });
    if (zero.load()) return fail(SL_EINVAL, "zero spin vector");
    // ordered on the system's stream; synchronised before the staging buffer is reused
    CK(cudaMemcpyAsync(dst, h, sizeof(double4) * s.n, cudaMemcpyHostToDevice, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    return SL_OK;
}

int download_vec(const sl::Sys &s, const double4 *src, double *dst) {
    double4 *h = stage_buffer(s);
    if (!h) return fail(SL_ENOMEM, "pinned staging buffer allocation failed");
    CK(cudaMemcpyAsync(h, src, sizeof(double4) * s.n, cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    const int32_t *orig = s.h_orig.data();
    parallel_chunks(s.n, [&](int64_t lo, int64_t hi) {
        for (int64_t i = lo; i < hi; ++i) {
            double *p = dst + 3 * (int64_t)orig[i];
            p[0] = h[i].x; p[1] = h[i].y; p[2] = h[i].z;
        }
    });
    return SL_OK;
}

__global__ void k_wrap_and_copy(double4 *pos, float4 *posf, const double4 *spin, float4 *spinf, int64_t n,
                                sl::BoxDev<double> b, int px, int py, int pz) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 r = pos[i];
    if (px) r.x = r.x - b.L[0] * floor(r.x / b.L[0]);
    if (py) r.y = r.y - b.L[1] * floor(r.y / b.L[1]);
    if (pz) r.z = r.z - b.L[2] * floor(r.z / b.L[2]);
    pos[i] = r;
    posf[i] = make_float4((float)r.x, (float)r.y, (float)r.z, 0.f);
    const double4 S = spin[i];
    spinf[i] = make_float4((float)S.x, (float)S.y, (float)S.z, 0.f);
}

int refresh_copies(sl::Sys &s) {
    if (s.n == 0) return SL_OK;
    k_wrap_and_copy<<<(unsigned)((s.n + 255) / 256), 256, 0, s.stream>>>(s.pos, s.posf, s.spin, s.spinf, s.n, s.boxd,
                                                                         s.per[0], s.per[1], s.per[2]);
    CK(cudaGetLastError());
    return SL_OK;
}

int capture_graph(sl::Sys &s, int k) {
    if (s.graph) {
        cudaGraphExecDestroy(s.graph);
        s.graph = nullptr;
    }
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
    for (int t = 0; t < k; ++t) enqueue_step(s);
    cudaError_t e = cudaStreamEndCapture(s.stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture");
    e = cudaGraphInstantiate(&s.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    s.graph_steps = k;
    return SL_OK;
}

// Launch shapes chosen by sl_autotune, per (device, precision, size bucket), shared by
// every system of the process so that later systems of a similar size start tuned.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, sl::LaunchCfg> g_tuned;

std::tuple<int, int, int> tune_key(const sl::Sys &s) {
    int bucket = 0;
    for (int64_t m = s.n; m > 1; m >>= 1) ++bucket;
    return std::make_tuple(s.device, s.prec, bucket);
}

void set_cfg(sl::Sys &s, const sl::LaunchCfg &c) {
    s.cfg = c;
    if (s.graph) {   // captured launches carry the old shapes
        cudaGraphExecDestroy(s.graph);
        s.graph = nullptr;
        s.graph_steps = 0;
    }
    ++s.capture_version;
}

}  // namespace

extern "C" {

void sl_default_options(sl_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = SL_PREC_FP64;
    o->seed = 1234;
    o->replica = 0;
    o->skin = 1.0;
    o->gamma_lattice_per_fs = 0.01;
    o->lambda_spin = 0.1;
    o->midpoint_iters = 0;
    o->midpoint_tol = 0.0;
    o->anderson_depth = 0;
    o->anderson_reg = 1e-10;
    o->nbr_cap_rad = 160;
    o->nbr_cap_ang = 64;
    o->steps_per_graph = 10;
    o->cuda_stream = nullptr;
    o->device = -1;
}

const char *sl_last_error(void) { return g_err.c_str(); }

int sl_create_system(const double *positions, const double *spins, const double box[3], const int32_t periodic[3],
                     const int32_t *species, int64_t n, const double *velocities, const sl_nep_params *params,
                     const sl_options *opt_in, sl_system **out) {
    NvtxRange nvtx_range("sl_create_system");
    using namespace sl;
    if (!out) return fail(SL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params || !box || !periodic) return fail(SL_EINVAL, "params, box and periodic are required");
    if (n < 0 || n >= (1LL << 30)) return fail(SL_EINVAL, "n = %lld out of range [0, 2^30)", (long long)n);
    if (n > 0 && (!positions || !spins || !species)) return fail(SL_EINVAL, "positions, spins, species required");
    if (params->n_species != NS || params->n_ch != NCH || params->l_max != 4 || params->basis_k != NK ||
        params->n_hidden != NH)
        return fail(SL_EINVAL, "model shape (%d species, %d channels, l_max %d, %d terms, %d hidden) not supported; "
                               "kernels are built for (2, 5, 4, 9, 30)",
                    params->n_species, params->n_ch, params->l_max, params->basis_k, params->n_hidden);
    if (!(params->rc_ang > 0 && params->rc_rad >= params->rc_ang))
        return fail(SL_EINVAL, "cutoffs must satisfy 0 < rc_ang <= rc_rad");
    if (!params->coeffs || !params->q_scaler || !params->w0 || !params->b0 || !params->w1 || !params->mass_amu ||
        !params->moment_muB)
        return fail(SL_EINVAL, "missing parameter array");
    sl_options opt;
    if (opt_in) opt = *opt_in;
    else sl_default_options(&opt);
    if (opt.precision != SL_PREC_FP64 && opt.precision != SL_PREC_MIXED) return fail(SL_EINVAL, "bad precision");
    if (!(opt.skin > 0)) return fail(SL_EINVAL, "skin must be positive");
    if (opt.midpoint_iters < 0 || opt.midpoint_iters > sl::MID_MAX_ITERS)
        return fail(SL_EINVAL, "midpoint_iters must lie in [0, %d]", sl::MID_MAX_ITERS);
    if (opt.anderson_depth < 0 || opt.anderson_depth > sl::AA_MAX_DEPTH)
        return fail(SL_EINVAL, "anderson_depth must lie in [0, %d]", sl::AA_MAX_DEPTH);
    if (!(opt.midpoint_tol >= 0) || !std::isfinite(opt.midpoint_tol) || !(opt.anderson_reg >= 0) ||
        !std::isfinite(opt.anderson_reg))
        return fail(SL_EINVAL, "midpoint_tol and anderson_reg must be finite and non-negative");
    if (opt.nbr_cap_rad < 1 || opt.nbr_cap_rad > 256 || opt.nbr_cap_ang < 1 || opt.nbr_cap_ang > opt.nbr_cap_rad)
        return fail(SL_EINVAL, "neighbour caps must satisfy 1 <= cap_ang <= cap_rad <= 256");
    if (opt.gamma_lattice_per_fs < 0 || opt.lambda_spin < 0) return fail(SL_EINVAL, "negative damping");
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0)) return fail(SL_EINVAL, "box lengths must be positive");
        if (periodic[a] && box[a] < 2.0 * (params->rc_rad + opt.skin))
            return fail(SL_EINVAL, "periodic box length %g below 2 (rc_rad + skin) = %g", box[a],
                        2.0 * (params->rc_rad + opt.skin));
    }
    for (int64_t i = 0; i < n; ++i)
        if (species[i] < 0 || species[i] >= NS) return fail(SL_EINVAL, "species[%lld] out of range", (long long)i);
    for (int t = 0; t < NS; ++t)
        if (!(params->mass_amu[t] > 0)) return fail(SL_EINVAL, "masses must be positive");

    int dev_count = 0;
    cudaError_t ce = cudaGetDeviceCount(&dev_count);
    if (ce != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(SL_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(ce));
    }

    if (opt.device >= dev_count) return fail(SL_EINVAL, "device %d not present (%d devices)", opt.device, dev_count);
    if (opt.device >= 0 && (ce = cudaSetDevice(opt.device)) != cudaSuccess) return cuda_fail(ce, "cudaSetDevice");
    sl_system *sys = new (std::nothrow) sl_system();
    static std::atomic<uint64_t> next_uid{1};
    if (sys) sys->s.uid = next_uid.fetch_add(1);
    if (!sys) return fail(SL_ENOMEM, "host allocation failed");
    Sys &s = sys->s;
    cudaGetDevice(&s.device);
    s.n = n;
    s.prec = opt.precision;
    s.seed = opt.seed;
    s.replica = opt.replica;
    s.skin = opt.skin;
    s.gamma = opt.gamma_lattice_per_fs;
    s.lambda = opt.lambda_spin;
    s.mid_iters = opt.midpoint_iters;
    s.mid_tol = opt.midpoint_tol;
    s.aa_depth = opt.midpoint_iters > 0 ? opt.anderson_depth : 0;
    s.aa_reg = opt.anderson_reg;
    s.cap = opt.nbr_cap_rad;
    s.cap_ang = opt.nbr_cap_ang;
    s.maskw = (s.cap + 31) / 32;
    s.steps_per_graph = opt.steps_per_graph < 0 ? 0 : opt.steps_per_graph;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(tune_key(s));
        if (it != g_tuned.end()) s.cfg = it->second;
    }
    fill_params(s.pd, params);
    fill_params(s.pf, params);
    for (int t = 0; t < NS; ++t) {
        s.mass[t] = params->mass_amu[t];
        s.moment[t] = params->moment_muB[t];
    }
    for (int a = 0; a < 3; ++a) {
        s.box[a] = box[a];
        s.per[a] = periodic[a] ? 1 : 0;
        s.boxd.L[a] = box[a];
        s.boxd.invL[a] = s.per[a] ? 1.0 / box[a] : 0.0;
        s.boxf.L[a] = (float)box[a];
        s.boxf.invL[a] = s.per[a] ? (float)(1.0 / box[a]) : 0.f;
    }
    s.cut_r2 = (params->rc_rad + s.skin) * (params->rc_rad + s.skin);
    s.cut_a2 = (params->rc_ang + s.skin) * (params->rc_ang + s.skin);
    nbr_setup(s);
    eval2_init();

    int rc = SL_OK;
    auto bail = [&](int code) {
        free_sys(s);
        delete sys;
        return code;
    };
    if (opt.cuda_stream) s.stream = (cudaStream_t)opt.cuda_stream;
    else {
        ce = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return bail(cuda_fail(ce, "cudaStreamCreate"));
        s.own_stream = true;
    }

    // internal order: species-major, then Morton order of the binning cells, then caller index
    std::vector<int32_t> order((size_t)n);
    {
        std::vector<uint64_t> key((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            uint32_t c[3];
            for (int a = 0; a < 3; ++a) {
                double x = positions[3 * i + a];
                if (s.per[a]) x = x - box[a] * std::floor(x / box[a]);
                const double w = box[a] / s.cells.nc[a];
                long ci = (long)std::floor(x / w);
                ci = std::min<long>(std::max<long>(ci, 0), s.cells.nc[a] - 1);
                c[a] = (uint32_t)ci;
            }
            key[i] = ((uint64_t)species[i] << 62) | morton3(c[0], c[1], c[2]);
            order[i] = (int32_t)i;
        }
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    std::vector<int32_t> inv((size_t)n), spec((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        inv[order[i]] = (int32_t)i;
        spec[i] = species[order[i]];
    }
    s.h_orig = order;   // host copy of the permutation for state transfers
    s.n_fe = 0;
    for (int64_t i = 0; i < n; ++i) s.n_fe += spec[i] == 0;

    const size_t N = (size_t)n;
    const size_t R = s.prec == SL_PREC_FP64 ? 8 : 4;
    s.qs = (n + 3) & ~(int64_t)3;
    if ((rc = dalloc(&s.pos, N)) || (rc = dalloc(&s.vel, N)) || (rc = dalloc(&s.spin, N)) ||
        (rc = dalloc(&s.spin_prev, N)) || (rc = dalloc(&s.F, N)) || (rc = dalloc(&s.H, N)) ||
        (rc = dalloc(&s.posref, N)) || (rc = dalloc(&s.posf, N)) || (rc = dalloc(&s.spinf, N)) ||
        (rc = dalloc(&s.species, N)) || (rc = dalloc(&s.orig, N)) || (rc = dalloc(&s.inv, N)) ||
        (rc = dalloc(&s.nbr, N * sl::nbr_stride(s.cap))) || (rc = dalloc(&s.rev, N * sl::nbr_stride(s.cap))) ||
        (rc = dalloc(&s.nbr_hash, N * sl::nbr_stride(s.cap))) ||
        (rc = dalloc(&s.cells.posf, N)) || (rc = dalloc(&s.cells.key, N)) || (rc = dalloc(&s.seg, N)) ||
        (rc = dalloc(&s.cells.count, (size_t)s.cells.ncell)) || (rc = dalloc(&s.cells.start, (size_t)s.cells.ncell + 1)) ||
        (rc = dalloc(&s.cells.fill, (size_t)s.cells.ncell)) || (rc = dalloc(&s.cells.atoms, N)) ||
        (rc = dalloc(&s.cells.of, N)) || (rc = dalloc(&s.cells.sub, (size_t)s.cells.ncell * 8)) || (rc = dalloc((char **)&s.q, R * DIM * (size_t)s.qs)) ||
        (rc = dalloc((char **)&s.bsum, R * NBREC * N)) || (rc = dalloc((char **)&s.fp, R * DIM * N)) ||
        (rc = dalloc((char **)&s.ei, R * N)) || (rc = dalloc((char **)&s.pairs, R * 8 * N * s.cap)) ||
        (rc = dalloc(&s.clj, N * (size_t)(s.cap + s.cap_ang))) || (rc = dalloc(&s.cls, N * (size_t)(s.cap + s.cap_ang))) ||
        (rc = dalloc(&s.cnt, N)) || (rc = dalloc(&s.cmask, N * (size_t)((s.cap + 31) / 32))) || (rc = dalloc((char **)&s.fown, R * 4 * N)) ||
        (rc = dalloc((char **)&s.gii, R * 4 * N)) || (rc = dalloc((char **)&s.wpart, R * 9 * N)) ||
        (rc = dalloc(&s.Fo, N)) || (rc = dalloc(&s.Ho, N)) || (rc = dalloc(&s.status, 1)) ||
        (rc = dalloc(&s.rebuild, 1)) || (rc = dalloc(&s.d_step, 2)) || (rc = dalloc(&s.d_par, 1)) ||
        (rc = dalloc(&s.red, 256 * 10 + 10)) || (rc = dalloc(&s.snap, 5 * N)) || (rc = dalloc(&s.d_builds, 1)))
        return bail(rc);
    if (s.prec == SL_PREC_MIXED && n > 0 && sl::make_q_tensor_map(s))
        return bail(fail(SL_ECUDA, "the TMA map of the descriptor array could not be encoded"));
    if (s.prec == SL_PREC_MIXED && n > 0 && sl::make_mlp_image(s))
        return bail(fail(SL_ENOMEM, "the network weights' operand images could not be made"));
    if (s.mid_iters > 0) {
        const size_t ring = (size_t)(s.aa_depth > 0 ? s.aa_depth + 1 : 0) * N;
        if ((rc = dalloc(&s.posmid, N)) || (rc = dalloc(&s.posmidf, N)) || (rc = dalloc(&s.mids, N)) ||
            (rc = dalloc(&s.midsf, N)) || (rc = dalloc(&s.mx, N)) || (rc = dalloc(&s.mg, N)) ||
            (rc = dalloc(&s.aax, ring)) || (rc = dalloc(&s.aag, ring)) ||
            (rc = dalloc(&s.aapart, sl::midpoint_scratch_doubles())) || (rc = dalloc(&s.md, 1)))
            return bail(rc);
        CK(cudaMemsetAsync(s.md, 0, sizeof(sl::MidDev), s.stream));
    }
    if ((ce = cudaMallocHost((void **)&s.h_par, sizeof(StepDev))) != cudaSuccess ||
        (ce = cudaMallocHost((void **)&s.h_status, sizeof(int))) != cudaSuccess ||
        (ce = cudaMallocHost((void **)&s.h_red, sizeof(double) * 10)) != cudaSuccess)
        return bail(fail(SL_ENOMEM, "pinned allocation failed: %s", cudaGetErrorString(ce)));

    // upload (internal order)
    {
        std::vector<double4> hp(N), hv(N), hs(N);
        for (size_t i = 0; i < N; ++i) {
            const int64_t c = order[i];
            hp[i] = make_double4(positions[3 * c], positions[3 * c + 1], positions[3 * c + 2], 0.0);
            const double sx = spins[3 * c], sy = spins[3 * c + 1], sz = spins[3 * c + 2];
            const double nn = std::sqrt(sx * sx + sy * sy + sz * sz);
            if (!(nn > 0) || !std::isfinite(nn)) return bail(fail(SL_EINVAL, "spin %lld is zero or non-finite", (long long)c));
            hs[i] = make_double4(sx / nn, sy / nn, sz / nn, 0.0);
            hv[i] = velocities ? make_double4(velocities[3 * c], velocities[3 * c + 1], velocities[3 * c + 2], 0.0)
                               : make_double4(0, 0, 0, 0);
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(positions[3 * c + a])) return bail(fail(SL_EINVAL, "non-finite position"));
        }
        // every copy on the system's stream (a non-blocking stream is not ordered
        // against the legacy default stream), then one synchronisation
        cudaStream_t st = s.stream;
        if ((ce = cudaMemcpyAsync(s.pos, hp.data(), sizeof(double4) * N, cudaMemcpyHostToDevice, st)) ||
            (ce = cudaMemcpyAsync(s.vel, hv.data(), sizeof(double4) * N, cudaMemcpyHostToDevice, st)) ||
            (ce = cudaMemcpyAsync(s.spin, hs.data(), sizeof(double4) * N, cudaMemcpyHostToDevice, st)) ||
            (ce = cudaMemcpyAsync(s.species, spec.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st)) ||
            (ce = cudaMemcpyAsync(s.orig, order.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st)) ||
            (ce = cudaMemcpyAsync(s.inv, inv.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, st)) ||
            (ce = cudaMemsetAsync(s.cells.count, 0, sizeof(int) * s.cells.ncell, st)) ||
            (ce = cudaMemsetAsync(s.cells.fill, 0, sizeof(int) * s.cells.ncell, st)) ||
            (ce = cudaMemsetAsync(s.status, 0, sizeof(int), st)) || (ce = cudaMemsetAsync(s.rebuild, 0, sizeof(int), st)) ||
            (ce = cudaMemsetAsync(s.d_step, 0, 2 * sizeof(unsigned long long), st)) ||
            (ce = cudaMemsetAsync(s.d_builds, 0, sizeof(unsigned long long), st)) ||
            (ce = cudaStreamSynchronize(st)))
            return bail(cuda_fail(ce, "upload"));
    }
    if (sl::solo_refresh(s)) return bail(fail(SL_ENOMEM, "the system's argument tables"));
    const double B0[3] = {0, 0, 0};
    if ((rc = upload_params(s, 1.0, 0.0, B0)) || (rc = refresh_copies(s)) || (rc = evaluate(s, true, true, false)) ||
        (rc = check_status(s)))
        return bail(rc);
    *out = sys;
    return SL_OK;
}

// State at the start of a stepping call, kept on the device so that a call that ends in
// a list overflow or a non-finite value leaves the system as it was before the call.
static int snapshot_state(sl::Sys &s) {
    const size_t N = (size_t)s.n;
    CK(cudaMemcpyAsync(s.snap, s.pos, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.snap + N, s.vel, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.snap + 2 * N, s.spin, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.snap + 3 * N, s.F, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.snap + 4 * N, s.H, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
    return SL_OK;
}

static int restore_state(sl::Sys &s) {
    const size_t N = (size_t)s.n;
    CK(cudaMemcpyAsync(s.pos, s.snap, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.vel, s.snap + N, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.spin, s.snap + 2 * N, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.F, s.snap + 3 * N, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(s.H, s.snap + 4 * N, sizeof(double4) * N, cudaMemcpyDeviceToDevice, s.stream));
    unsigned long long st[2] = {s.step, s.step};
    CK(cudaMemcpyAsync(s.d_step, st, sizeof st, cudaMemcpyHostToDevice, s.stream));
    CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
    int r2;
    if ((r2 = refresh_copies(s))) return r2;
    sl::launch_rebuild(s, false);
    CK(cudaStreamSynchronize(s.stream));
    return SL_OK;
}

// ------------------------------------------------------------------ coloured spin sweep
// Squared minimum-image distance with one rounding per operation and no fused multiply-add
// (the neighbour-list arithmetic): each intermediate goes through a volatile so that no
// compiler contraction can change a borderline decision.
static double exact_d2_host(const double *a, const double *b, const double *L, const int *per) {
    volatile double t[3];
    for (int k = 0; k < 3; ++k) {
        volatile double u = b[k] - a[k];
        if (per[k]) {
            volatile double q = std::rint(u / L[k]);
            volatile double m = L[k] * q;
            u = u - m;
        }
        t[k] = u;
    }
    volatile double xx = t[0] * t[0], yy = t[1] * t[1], zz = t[2] * t[2];
    volatile double sxy = xx + yy;
    return sxy + zz;
}

// Greedy colouring, in caller index order, of the graph joining atoms closer than 2 rc_rad:
// colour(i) = the smallest c used by no conflicting atom of lower caller index.  Positions
// are the device state (internal order); the colours go back to the device in internal order.
static int colour_atoms(sl::Sys &s) {
    const int64_t n = s.n;
    std::vector<double4> h((size_t)n);
    CK(cudaMemcpyAsync(h.data(), s.pos, sizeof(double4) * n, cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    // caller-order coordinates
    std::vector<double> x((size_t)(3 * n));
    for (int64_t k = 0; k < n; ++k) {
        const int64_t c = s.h_orig[(size_t)k];
        x[3 * c] = h[k].x; x[3 * c + 1] = h[k].y; x[3 * c + 2] = h[k].z;
    }
    const double cut = 2.0 * s.pd.rc_r, cut2 = cut * cut;
    // cell list with cells of at least the conflict radius (all cells when a dimension has fewer than 3)
    int nc[3];
    for (int a = 0; a < 3; ++a) nc[a] = std::max(1, (int)std::floor(s.box[a] / (cut * (1.0 + 1e-9))));
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    std::vector<int64_t> cstart((size_t)ncell + 1, 0), catoms((size_t)n);
    std::vector<int32_t> cof((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * i + a];
            if (s.per[a]) v = v - s.box[a] * std::floor(v / s.box[a]);
            ci[a] = std::min(std::max((int)std::floor(v / (s.box[a] / nc[a])), 0), nc[a] - 1);
        }
        cof[i] = (int32_t)(((int64_t)ci[2] * nc[1] + ci[1]) * nc[0] + ci[0]);
        cstart[(size_t)cof[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        std::vector<int64_t> fill(cstart.begin(), cstart.end() - 1);
        for (int64_t i = 0; i < n; ++i) catoms[(size_t)fill[(size_t)cof[i]]++] = i;
    }
    std::vector<int32_t> col((size_t)n, -1);
    std::vector<char> used;
    int32_t ncol = 0;
    std::vector<int32_t> seen;
    for (int64_t i = 0; i < n; ++i) {
        const int32_t cc = cof[i];
        const int ci[3] = {(int)(cc % nc[0]), (int)((cc / nc[0]) % nc[1]), (int)(cc / ((int64_t)nc[0] * nc[1]))};
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            if (s.per[a] && nc[a] < 3) { lo[a] = 0; hi[a] = nc[a] - 1; }
            else if (s.per[a]) { lo[a] = ci[a] - 1; hi[a] = ci[a] + 1; }
            else { lo[a] = std::max(ci[a] - 1, 0); hi[a] = std::min(ci[a] + 1, nc[a] - 1); }
        }
        seen.clear();
        for (int z = lo[2]; z <= hi[2]; ++z)
            for (int y = lo[1]; y <= hi[1]; ++y)
                for (int xx = lo[0]; xx <= hi[0]; ++xx) {
                    const int wx = (xx % nc[0] + nc[0]) % nc[0], wy = (y % nc[1] + nc[1]) % nc[1],
                              wz = (z % nc[2] + nc[2]) % nc[2];
                    const int64_t c = ((int64_t)wz * nc[1] + wy) * nc[0] + wx;
                    for (int64_t p = cstart[(size_t)c]; p < cstart[(size_t)c + 1]; ++p) {
                        const int64_t j = catoms[(size_t)p];
                        if (j >= i) continue;
                        if (exact_d2_host(&x[3 * i], &x[3 * j], s.box, s.per) < cut2) seen.push_back(col[(size_t)j]);
                    }
                }
        if ((int64_t)used.size() < (int64_t)ncol + 1) used.resize((size_t)ncol + 1, 0);
        for (int32_t c : seen) used[(size_t)c] = 1;
        int32_t c = 0;
        while (c < ncol && used[(size_t)c]) ++c;
        col[(size_t)i] = c;
        ncol = std::max(ncol, c + 1);
        for (int32_t q : seen) used[(size_t)q] = 0;
    }
    std::vector<int32_t> hint((size_t)n);
    for (int64_t k = 0; k < n; ++k) hint[(size_t)k] = col[(size_t)s.h_orig[(size_t)k]];
    CK(cudaMemcpyAsync(s.colour, hint.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    s.last_colours = ncol;
    return SL_OK;
}

// One step with the coloured sweep: lattice first half (spins untouched), conditional list
// rebuild, colouring at the new positions, 2C sub-steps (evaluation + half-step rotation of one
// colour, colours 0..C-1 then C-1..0), the final evaluation and the lattice kick.  Driven from
// the host: the colouring and the number of sub-steps depend on the positions.
static int sweep_step(sl::Sys &s) {
    sl::launch_first_half(s);
    sl::launch_rebuild(s, true);
    int rc;
    if ((rc = colour_atoms(s))) return rc;
    const int C = s.last_colours;
    for (int pass = 0; pass < 2 * C; ++pass) {
        sl::launch_eval(s, false);
        sl::launch_sweep_rotate(s, pass < C ? pass : 2 * C - 1 - pass);
    }
    sl::launch_eval(s, false);
    sl::launch_second_half_nospin(s);
    CK(cudaGetLastError());
    s.sweep_evaluations += 2 * C + 1;
    s.n_launches += sl::KERNELS_PER_STEP + (int64_t)2 * C * 5;
    return SL_OK;
}

// Queue n_steps steps on the system's stream: captured graphs of steps_per_graph steps,
// then single steps for the remainder.
static int queue_steps(sl::Sys &s, int64_t n_steps) {
    int rc;
    int64_t left = n_steps;
    const int k = s.steps_per_graph;
    if (k > 0 && left >= k) {
        if (!s.graph || s.graph_steps != k)
            if ((rc = capture_graph(s, k))) return rc;
        while (left >= k) {
            CK(cudaGraphLaunch(s.graph, s.stream));
            left -= k;
        }
    }
    for (; left > 0; --left) enqueue_step(s);
    CK(cudaGetLastError());
    s.n_launches += n_steps * kernels_per_step(s);
    return SL_OK;
}

// Status of the queued steps; on a list overflow or a non-finite value the state goes
// back to the snapshot and the error names the step it was restored to.
static int finish_steps(sl::Sys &s, int64_t n_steps, const char *who) {
    const int rc = check_status(s);
    if (rc == SL_ENBR_OVERFLOW || rc == SL_ENONFINITE) {
        const std::string msg = g_err;
        int r2;
        if ((r2 = restore_state(s))) return r2;
        return fail(rc, "%s%s; state restored to step %llu", who, msg.c_str(), (unsigned long long)s.step);
    }
    if (rc) return rc;
    s.step += (uint64_t)n_steps;
    return SL_OK;
}

int sl_step(sl_system *sys, int64_t n_steps, double dt, double T, const double B[3]) {
    NvtxRange nvtx_range("sl_step");
    if (!sys || !B) return fail(SL_EINVAL, "NULL argument");
    if (n_steps < 0 || !(dt > 0) || !(T >= 0) || !std::isfinite(dt) || !std::isfinite(T))
        return fail(SL_EINVAL, "bad step arguments");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    int rc;
    if ((rc = upload_params(s, dt, T, B))) return rc;
    for (int c = 0; c < 3; ++c) s.B[c] = B[c];
    if (n_steps == 0 || s.n == 0) {
        s.step += (uint64_t)n_steps;
        return SL_OK;
    }
    if ((rc = snapshot_state(s))) return rc;
    if (s.sts) {
        for (int64_t t = 0; t < n_steps; ++t)
            if ((rc = sweep_step(s))) return rc;
    } else if ((rc = queue_steps(s, n_steps))) {
        return rc;
    }
    return finish_steps(s, n_steps, "");
}

int sl_energy_forces_fields(sl_system *sys, double *energy, double *forces, double *fields, double *virial) {
    NvtxRange nvtx_range("sl_energy_forces_fields");
    if (!sys) return fail(SL_EINVAL, "NULL system");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    if (s.n == 0) {
        if (energy) *energy = 0.0;
        if (virial) std::memset(virial, 0, 9 * sizeof(double));
        return SL_OK;
    }
    int rc;
    CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
    if ((rc = evaluate(s, false, false, virial != nullptr))) return rc;
    if ((rc = check_status(s))) return rc;
    double E, W[9];
    if (sl::reduce_energy_virial(s, &E, W, virial != nullptr)) return fail(SL_ECUDA, "reduction failed");
    if (energy) *energy = E;
    if (virial) std::memcpy(virial, W, sizeof W);
    if (forces && (rc = download_vec(s, s.Fo, forces))) return rc;
    if (fields && (rc = download_vec(s, s.Ho, fields))) return rc;
    return SL_OK;
}

int sl_get_descriptors(sl_system *sys, double *q, double *atom_energy) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    if (s.n == 0) return SL_OK;
    int rc;
    if ((rc = evaluate(s, false, false, false))) return rc;
    const size_t N = (size_t)s.n, R = s.prec == 0 ? 8 : 4, QS = (size_t)s.qs;
    std::vector<char> hq(R * sl::DIM * QS), he(R * N);
    std::vector<int32_t> orig(N);
    CK(cudaMemcpyAsync(hq.data(), s.q, hq.size(), cudaMemcpyDeviceToHost, s.stream));
    CK(cudaMemcpyAsync(he.data(), s.ei, he.size(), cudaMemcpyDeviceToHost, s.stream));
    CK(cudaMemcpyAsync(orig.data(), s.orig, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    auto get = [&](const std::vector<char> &b, size_t idx) {
        return R == 8 ? ((const double *)b.data())[idx] : (double)((const float *)b.data())[idx];
    };
    for (size_t i = 0; i < N; ++i) {
        if (q)
            for (int v = 0; v < sl::DIM; ++v) q[(size_t)orig[i] * sl::DIM + v] = get(hq, (size_t)v * QS + i);
        if (atom_energy) atom_energy[orig[i]] = get(he, i);
    }
    return SL_OK;
}

int sl_get_state(const sl_system *sys, double *pos, double *vel, double *spins, double *forces, double *fields,
                 double *ref, uint64_t *step) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    const sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    int rc;
    if (s.n > 0) {
        if (pos && (rc = download_vec(s, s.pos, pos))) return rc;
        if (vel && (rc = download_vec(s, s.vel, vel))) return rc;
        if (spins && (rc = download_vec(s, s.spin, spins))) return rc;
        if (forces && (rc = download_vec(s, s.F, forces))) return rc;
        if (fields && (rc = download_vec(s, s.H, fields))) return rc;
        if (ref && (rc = download_vec(s, s.posref, ref))) return rc;
    }
    if (step) *step = s.step;
    return SL_OK;
}

int sl_set_state(sl_system *sys, const double *pos, const double *vel, const double *spins, const double *forces,
                 const double *fields, const double *ref, uint64_t step) {
    NvtxRange nvtx_range("sl_set_state");
    if (!sys) return fail(SL_EINVAL, "NULL system");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    if (s.n > 0 && (!pos || !vel || !spins)) return fail(SL_EINVAL, "positions, velocities and spins are required");
    if ((forces == nullptr) != (fields == nullptr)) return fail(SL_EINVAL, "give both forces and fields or neither");
    int rc;
    CK(cudaStreamSynchronize(s.stream));
    if (s.n > 0) {
        for (int64_t i = 0; i < 3 * s.n; ++i)
            if (!std::isfinite(pos[i]) || !std::isfinite(vel[i]) || !std::isfinite(spins[i]) ||
                (ref && !std::isfinite(ref[i])))
                return fail(SL_EINVAL, "non-finite state value");
        // unit spins are normalised on entry; in the longitudinal mode their lengths are state
        if ((rc = upload_vec(s, s.vel, vel, false)) || (rc = upload_vec(s, s.spin, spins, !s.lng))) return rc;
        // lists from the reference positions (k_finish records them as the new reference)
        if ((rc = upload_vec(s, s.pos, ref ? ref : pos, false)) || (rc = refresh_copies(s))) return rc;
        CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
        sl::launch_rebuild(s, false);
        s.n_builds++;
        if (ref && ((rc = upload_vec(s, s.pos, pos, false)) || (rc = refresh_copies(s)))) return rc;
    }
    s.step = step;
    unsigned long long st[2] = {step, step};
    CK(cudaMemcpyAsync(s.d_step, st, sizeof st, cudaMemcpyHostToDevice, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    if (s.n > 0) {
        if (forces) {
            if ((rc = upload_vec(s, s.F, forces, false)) || (rc = upload_vec(s, s.H, fields, false))) return rc;
        } else if ((rc = evaluate(s, false, true, false))) {
            return rc;
        }
    }
    CK(cudaGetLastError());
    return check_status(s);
}

int sl_get_neighbors(sl_system *sys, int32_t cap, int32_t *counts_rad, int32_t *lists_rad, int32_t *counts_ang,
                     int32_t *lists_ang) {
    if (!sys || cap < 0) return fail(SL_EINVAL, "bad arguments");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    if (s.n == 0) return SL_OK;
    CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
    sl::launch_rebuild(s, false);
    s.n_builds++;
    int rc = check_status(s);
    if (rc) return rc;
    const size_t N = (size_t)s.n;
    std::vector<int32_t> nbr(N * sl::nbr_stride(s.cap)), orig(N);
    std::vector<int4> seg(N);
    CK(cudaMemcpyAsync(nbr.data(), s.nbr, sizeof(int32_t) * N * sl::nbr_stride(s.cap), cudaMemcpyDeviceToHost,
                       s.stream));
    CK(cudaMemcpyAsync(orig.data(), s.orig, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, s.stream));
    CK(cudaMemcpyAsync(seg.data(), s.seg, sizeof(int4) * N, cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    bool over = false;
    for (size_t i = 0; i < N; ++i) {
        const int c = orig[i];
        std::vector<int32_t> rad, ang;
        for (int t = 0; t < seg[i].w; ++t) {
            const int32_t j = orig[nbr[(size_t)i * sl::nbr_stride(s.cap) + t]];
            rad.push_back(j);
            if (t < seg[i].y) ang.push_back(j);
        }
        std::sort(rad.begin(), rad.end());
        std::sort(ang.begin(), ang.end());
        if (counts_rad) counts_rad[c] = (int32_t)rad.size();
        if (counts_ang) counts_ang[c] = (int32_t)ang.size();
        if ((int)rad.size() > cap) over = true;
        if (lists_rad)
            for (size_t t = 0; t < rad.size() && (int)t < cap; ++t) lists_rad[(size_t)c * cap + t] = rad[t];
        if (lists_ang)
            for (size_t t = 0; t < ang.size() && (int)t < cap; ++t) lists_ang[(size_t)c * cap + t] = ang[t];
    }
    if (over) return fail(SL_EINVAL, "a list is longer than the output capacity %d", cap);
    return SL_OK;
}

int sl_get_info(const sl_system *sys, int64_t *n_atoms, int32_t *precision, int64_t *n_builds,
                int64_t *n_launches) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    const sl::Sys &s = sys->s;
    if (n_atoms) *n_atoms = s.n;
    if (precision) *precision = s.prec;
    if (n_builds) {
        unsigned long long b = 0;
        cudaSetDevice(s.device);
        CK(cudaMemcpyAsync(&b, s.d_builds, sizeof b, cudaMemcpyDeviceToHost, s.stream));
        CK(cudaStreamSynchronize(s.stream));
        *n_builds = (int64_t)b;
    }
    if (n_launches) *n_launches = s.n_launches;
    return SL_OK;
}

int sl_autotune(sl_system *sys, int32_t repeats, int32_t *chosen, double *eval_ms_before, double *eval_ms_after) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    if (repeats < 1 || repeats > 1000) return fail(SL_EINVAL, "repeats must lie in [1, 1000]");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    const sl::LaunchCfg before = s.cfg;
    auto report = [&](const sl::LaunchCfg &c) {
        if (chosen) {
            const int q = sl::default_quad_block(s.prec);
            chosen[0] = c.crad_block;
            chosen[1] = c.ang_block ? c.ang_block : q;
            chosen[2] = c.bwd_block ? c.bwd_block : q;
            chosen[3] = c.mlp_ctas_per_sm;
        }
    };
    if (s.n == 0) {
        report(s.cfg);
        if (eval_ms_before) *eval_ms_before = 0.0;
        if (eval_ms_after) *eval_ms_after = 0.0;
        return SL_OK;
    }
    // evaluation kernel groups timed by launch_eval's events: 1 radial (with compaction),
    // 2 angular forward, 3 network, 4 backward
    auto time_cfg = [&](const sl::LaunchCfg &c, double ms[5]) -> int {
        s.cfg = c;
        std::vector<cudaEvent_t> ev(6 * (size_t)repeats);
        for (auto &e : ev) CK(cudaEventCreate(&e));
        sl::launch_eval(s, false);   // warm-up
        for (int r = 0; r < repeats; ++r) sl::launch_eval(s, false, ev.data() + 6 * r);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s.stream));
        for (int g = 0; g < 5; ++g) {
            std::vector<float> t((size_t)repeats);
            for (int r = 0; r < repeats; ++r) CK(cudaEventElapsedTime(&t[r], ev[6 * r + g], ev[6 * r + g + 1]));
            std::sort(t.begin(), t.end());
            ms[g] = t[(size_t)repeats / 2];
        }
        for (auto &e : ev) cudaEventDestroy(e);
        return SL_OK;
    };
    // Candidate shapes: block size (half or full default) x register budget (the default, or
    // the kernel's variant, mixed precision only); network CTAs per SM 1 or 2.  Each kernel's
    // time depends on its own shape only, so one evaluation per candidate times every kernel
    // and each kernel takes its fastest.
    const int q = sl::default_quad_block(s.prec);
    const int ncand = s.prec == 0 ? 2 : 4;
    sl::LaunchCfg cand[4];
    for (int c = 0; c < ncand; ++c) {
        const bool half = (c & 1) == 0, var = c >= 2;
        cand[c].crad_block = half ? 64 : 128;
        cand[c].ang_block = half ? q / 2 : q;
        cand[c].bwd_block = half ? q / 2 : q;
        cand[c].mlp_ctas_per_sm = half ? 1 : 2;
        cand[c].crad_minb = var ? 3 : 0;
        cand[c].ang_minb = var ? 1 : 0;
        cand[c].bwd_minb = var ? 3 : 0;
    }
    double ms0[5], msc[4][5];
    int rc;
    // the shapes must not change any result: the forces and fields gathered after each
    // candidate's evaluations are compared bit for bit with those of the starting shape
    double4 *ref = nullptr;
    int *diff = nullptr;
    if ((rc = dalloc(&ref, 2 * (size_t)s.n)) || (rc = dalloc(&diff, 1))) {
        if (ref) cudaFree(ref);
        return rc;
    }
    auto cleanup = [&]() {
        cudaFree(ref);
        cudaFree(diff);
        s.cfg = before;
    };
    if ((rc = time_cfg(before, ms0))) {
        cleanup();
        return rc;
    }
    sl::launch_gather(s, false);
    CK(cudaMemcpyAsync(ref, s.Fo, sizeof(double4) * s.n, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemcpyAsync(ref + s.n, s.Ho, sizeof(double4) * s.n, cudaMemcpyDeviceToDevice, s.stream));
    CK(cudaMemsetAsync(diff, 0, sizeof(int), s.stream));
    for (int c = 0; c < ncand; ++c) {
        if ((rc = time_cfg(cand[c], msc[c]))) {
            cleanup();
            return rc;
        }
        sl::launch_gather(s, false);
        sl::launch_compare_bits(s, ref, diff);
    }
    int h_diff = 0;
    CK(cudaMemcpyAsync(&h_diff, diff, sizeof(int), cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    cleanup();
    if (h_diff) return fail(SL_EINTERNAL, "a launch shape changed the forces or fields");
    auto argmin = [&](int g) {
        int m = 0;
        for (int c = 1; c < ncand; ++c)
            if (msc[c][g] < msc[m][g]) m = c;
        return m;
    };
    const int kc = argmin(1), ka = argmin(2), km = argmin(3), kb = argmin(4);
    sl::LaunchCfg best;
    best.crad_block = cand[kc].crad_block; best.crad_minb = cand[kc].crad_minb;
    best.ang_block = cand[ka].ang_block; best.ang_minb = cand[ka].ang_minb;
    best.mlp_ctas_per_sm = s.prec != 0 ? cand[km].mlp_ctas_per_sm : before.mlp_ctas_per_sm;
    best.bwd_block = cand[kb].bwd_block; best.bwd_minb = cand[kb].bwd_minb;
    double after = msc[kc][1] + msc[ka][2] + msc[s.prec != 0 ? km : 0][3] + msc[kb][4], b0 = 0.0;
    for (int g = 1; g < 5; ++g) b0 += ms0[g];
    for (int c = 0; c < 4; ++c)
        for (int g = 0; g < 4; ++g) s.tune_ms[c][g] = c < ncand ? msc[c][g + 1] : -1.0;
    s.cfg = before;
    set_cfg(s, best);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[tune_key(s)] = best;
    }
    report(best);
    if (eval_ms_before) *eval_ms_before = b0;
    if (eval_ms_after) *eval_ms_after = after;
    return SL_OK;
}

int sl_get_launch_config(const sl_system *sys, int32_t *cfg, double *landscape) {
    if (!sys || !cfg) return fail(SL_EINVAL, "NULL argument");
    const sl::Sys &s = sys->s;
    const int q = sl::default_quad_block(s.prec);
    const sl::LaunchCfg &c = s.cfg;
    const int32_t v[8] = {c.crad_block, c.crad_minb, c.ang_block ? c.ang_block : q, c.ang_minb,
                          c.bwd_block ? c.bwd_block : q, c.bwd_minb, c.mlp_ctas_per_sm, 0};
    for (int k = 0; k < 8; ++k) cfg[k] = v[k];
    if (landscape)
        for (int k = 0; k < 16; ++k) landscape[k] = s.tune_ms[k / 4][k % 4];
    return SL_OK;
}

int sl_set_atom_fields(sl_system *sys, const double *B_atoms) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    // a captured step graph holds the field pointer: drop it whenever the pointer changes
    auto drop_graph = [&]() {
        if (s.graph) {
            cudaGraphExecDestroy(s.graph);
            s.graph = nullptr;
            s.graph_steps = 0;
        }
        ++s.capture_version;
    };
    if (!B_atoms) {
        if (s.Bat) {
            CK(cudaStreamSynchronize(s.stream));
            cudaFree(s.Bat);
            s.Bat = nullptr;
            drop_graph();
            if (sl::solo_refresh(s)) return fail(SL_ECUDA, "the system's argument tables");
        }
        return SL_OK;
    }
    for (int64_t k = 0; k < 3 * s.n; ++k)
        if (!std::isfinite(B_atoms[k])) return fail(SL_EINVAL, "non-finite per-atom field entry %lld", (long long)k);
    int rc;
    if (!s.Bat) {
        if ((rc = dalloc(&s.Bat, (size_t)(s.n > 0 ? s.n : 1)))) return rc;
        drop_graph();
        if (sl::solo_refresh(s)) return fail(SL_ECUDA, "the system's argument tables");
    }
    if (s.n > 0 && (rc = upload_vec(s, s.Bat, B_atoms, false))) return rc;
    return SL_OK;
}

int sl_set_spin_sweep(sl_system *sys, int32_t enable) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    sl::Sys &s = sys->s;
    if (enable && s.mid_iters > 0) return fail(SL_EINVAL, "the coloured sweep does not combine with the midpoint update");
    if (enable && s.lng) return fail(SL_EINVAL, "the coloured sweep does not combine with the longitudinal mode");
    cudaSetDevice(s.device);
    CK(cudaStreamSynchronize(s.stream));
    if (enable && !s.colour && s.n > 0) {
        int rc;
        if ((rc = dalloc(&s.colour, (size_t)s.n))) return rc;
    }
    s.sts = enable ? 1 : 0;
    return upload_params(s, s.last_dt, s.last_T, s.B);
}

int sl_get_sweep_colours(const sl_system *sys, int32_t *colours, int32_t *n_colours, int64_t *evaluations) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    const sl::Sys &s = sys->s;
    if (n_colours) *n_colours = s.last_colours;
    if (evaluations) *evaluations = s.sweep_evaluations;
    if (colours && s.n > 0) {
        if (!s.colour || s.last_colours == 0) return fail(SL_EINVAL, "no coloured step has been taken");
        cudaSetDevice(s.device);
        std::vector<int32_t> h((size_t)s.n);
        CK(cudaMemcpyAsync(h.data(), s.colour, sizeof(int32_t) * s.n, cudaMemcpyDeviceToHost, s.stream));
        CK(cudaStreamSynchronize(s.stream));
        for (int64_t k = 0; k < s.n; ++k) colours[s.h_orig[(size_t)k]] = h[(size_t)k];
    }
    return SL_OK;
}

int sl_set_longitudinal(sl_system *sys, int32_t enable, double alpha, const double *landau) {
    if (!sys) return fail(SL_EINVAL, "NULL system");
    sl::Sys &s = sys->s;
    if (enable && s.sts) return fail(SL_EINVAL, "the longitudinal mode does not combine with the coloured sweep");
    if (enable) {
        if (!(alpha >= 0) || !std::isfinite(alpha)) return fail(SL_EINVAL, "alpha must be finite and >= 0");
        if (s.mid_iters > 0) return fail(SL_EINVAL, "the longitudinal mode does not combine with the midpoint update");
        if (landau)
            for (int k = 0; k < 2 * sl::NS; ++k)
                if (!std::isfinite(landau[k])) return fail(SL_EINVAL, "non-finite Landau coefficient");
    }
    cudaSetDevice(s.device);
    CK(cudaStreamSynchronize(s.stream));
    const bool leaving = s.lng && !enable;
    s.lng = enable ? 1 : 0;
    s.lng_alpha = enable ? alpha : 0.0;
    for (int t = 0; t < sl::NS; ++t)
        for (int c = 0; c < 2; ++c)
            s.landau[t][c] = (enable && landau) ? landau[2 * t + c] : 0.0;
    int rc;
    if ((rc = upload_params(s, s.last_dt, s.last_T, s.B))) return rc;
    if (s.n == 0) return SL_OK;
    CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
    if (leaving) sl::launch_normalise_spins(s);
    // the carried forces and fields of the current state under the new energy
    if ((rc = evaluate(s, false, true, false))) return rc;
    return check_status(s);
}

int sl_texture_map(sl_system *sys, int32_t normal_axis, double cell, int32_t *n_a, int32_t *n_b, double *m,
                   double *Q) {
    if (!sys || !n_a || !n_b) return fail(SL_EINVAL, "NULL argument");
    if (normal_axis < 0 || normal_axis > 2) return fail(SL_EINVAL, "normal_axis must be 0, 1 or 2");
    if (!(cell > 0) || !std::isfinite(cell)) return fail(SL_EINVAL, "cell must be positive");
    sl::Sys &s = sys->s;
    int na, nb;
    sl::texture_grid(s, normal_axis, cell, &na, &nb);
    if ((int64_t)na * nb > (int64_t)1 << 28) return fail(SL_EINVAL, "texture grid of %d x %d cells is too large", na, nb);
    *n_a = na;
    *n_b = nb;
    if (!m && !Q) return SL_OK;
    cudaSetDevice(s.device);
    const cudaError_t e = sl::launch_texture(s, normal_axis, cell, m, Q);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(SL_ENOMEM, "texture scratch: %s", cudaGetErrorString(e))
                                              : cuda_fail(e, "texture diagnostics");
    }
    return SL_OK;
}

int sl_get_midpoint_evaluations(const sl_system *sys, int64_t *evaluations) {
    if (!sys || !evaluations) return fail(SL_EINVAL, "NULL argument");
    const sl::Sys &s = sys->s;
    *evaluations = 0;
    if (s.mid_iters <= 0 || !s.md) return SL_OK;
    unsigned long long v = 0;
    cudaSetDevice(s.device);
    CK(cudaMemcpyAsync(&v, reinterpret_cast<const char *>(s.md) + offsetof(sl::MidDev, iters), sizeof v,
                       cudaMemcpyDeviceToHost, s.stream));
    CK(cudaStreamSynchronize(s.stream));
    *evaluations = (int64_t)v;
    return SL_OK;
}

int64_t sl_estimate_device_bytes(int64_t n, const sl_options *opt_in) {
    sl_options opt;
    if (opt_in) opt = *opt_in;
    else sl_default_options(&opt);
    if (n < 0) return -1;
    const int64_t R = opt.precision == SL_PREC_FP64 ? 8 : 4;
    const int64_t cap = opt.nbr_cap_rad, ca = opt.nbr_cap_ang;
    int64_t per = 7 * 32 + 2 * 16                      // state (double4) and FP32 copies
                  + 3 * 4 + 4 + 16 + 16 + 4            // species, caller index maps, list segments, cell copies
                  + 6 * sl::nbr_stride((int)cap)     // candidate lists, reverse slots and index hashes (1 byte each)
                  + 6 * (ca + cap) + 16                // compact rows, counts
                  + 4 * ((cap + 31) / 32)              // in-cutoff slot mask
                  + R * (2 * sl::DIM + sl::NBREC + 1 + 9) // q, Fp, angular sums, E_i, virial parts
                  + R * 8 * cap + 2 * R * 4            // pair records, per-atom sums
                  + 2 * 32 + 5 * 32 + 4 * 4;           // evaluation outputs, snapshot, cell arrays
    if (opt.midpoint_iters > 0)                        // midpoint positions and spins, iterate, image, rings
        per += 4 * 32 + 2 * 16 + (opt.anderson_depth > 0 ? 2 * 32 * (opt.anderson_depth + 1) : 0);
    return n * per + (1 << 20);
}

int sl_step_profiled(sl_system *sys, int64_t n_steps, double dt, double T, const double B[3], double *kernel_ms) {
    NvtxRange nvtx_range("sl_step_profiled");
    if (!sys || !B || !kernel_ms) return fail(SL_EINVAL, "NULL argument");
    if (sys->s.sts) return fail(SL_EINVAL, "per-kernel profiling does not cover the coloured sweep");
    if (n_steps < 0 || !(dt > 0) || !(T >= 0)) return fail(SL_EINVAL, "bad step arguments");
    sl::Sys &s = sys->s;
    cudaSetDevice(s.device);
    for (int k = 0; k < SL_NKERNELS; ++k) kernel_ms[k] = 0.0;
    int rc;
    if ((rc = upload_params(s, dt, T, B))) return rc;
    for (int c = 0; c < 3; ++c) s.B[c] = B[c];
    if (s.n == 0 || n_steps == 0) { s.step += (uint64_t)n_steps; return SL_OK; }
    CK(cudaMemsetAsync(s.status, 0, sizeof(int), s.stream));
    // events per step: before first half, before rebuild, before each evaluation kernel (5), after the
    // last one, after second half, and after the rebuild (e[9]): in the midpoint mode the iteration
    // runs between e[9] and e[2] and counts as spin update (second-half group)
    const int EV = 10;
    std::vector<cudaEvent_t> ev((size_t)EV * n_steps);
    for (auto &e : ev) CK(cudaEventCreate(&e));
    for (int64_t t = 0; t < n_steps; ++t) {
        cudaEvent_t *e = ev.data() + EV * t;
        CK(cudaEventRecord(e[0], s.stream));
        sl::launch_first_half(s);
        CK(cudaEventRecord(e[1], s.stream));
        sl::launch_rebuild(s, true);
        CK(cudaEventRecord(e[9], s.stream));
        sl::launch_midpoint(s);
        sl::launch_eval(s, false, e + 2);   // e[2..7]
        if (s.mid_iters > 0) sl::launch_second_half_nospin(s);
        else sl::launch_second_half(s);
        CK(cudaEventRecord(e[8], s.stream));
    }
    CK(cudaGetLastError());
    s.n_launches += n_steps * kernels_per_step(s);
    rc = check_status(s);
    for (int64_t t = 0; t < n_steps && rc == SL_OK; ++t) {
        cudaEvent_t *e = ev.data() + EV * t;
        float ms;
        CK(cudaEventElapsedTime(&ms, e[0], e[1]));
        kernel_ms[SL_K_FIRST_HALF] += ms;
        CK(cudaEventElapsedTime(&ms, e[1], e[9]));
        kernel_ms[SL_K_REBUILD] += ms;
        CK(cudaEventElapsedTime(&ms, e[9], e[2]));
        kernel_ms[SL_K_SECOND_HALF] += ms;
        for (int k = SL_K_COMPACT; k <= SL_K_SECOND_HALF; ++k) {
            CK(cudaEventElapsedTime(&ms, e[k], e[k + 1]));
            kernel_ms[k] += ms;
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    s.step += (uint64_t)n_steps;
    return SL_OK;
}

int sl_measure_fma_peak(int32_t precision, double *flops, double *ms) {
    if (!flops) return fail(SL_EINVAL, "NULL argument");
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(SL_ECUDA, "no usable CUDA device");
    }
    double t = 0;
    if (sl::measure_fma_peak(precision, flops, &t)) return fail(SL_ECUDA, "peak kernel failed");
    if (ms) *ms = t;
    return SL_OK;
}

void *sl_get_stream(const sl_system *sys) { return sys ? (void *)sys->s.stream : nullptr; }

void sl_destroy_system(sl_system *sys) {
    if (!sys) return;
    cudaSetDevice(sys->s.device);
    if (sys->s.stream) cudaStreamSynchronize(sys->s.stream);
    free_sys(sys->s);
    delete sys;
}

// ---------------------------------------------------------------- batches
// precision of the batch's occupied slots (-1: none)
static int batch_precision(const sl_batch *b, int skip = -1) {
    for (int i = 0; i < (int)b->sys.size(); ++i)
        if (i != skip && b->sys[i]) return b->sys[i]->s.prec;
    return -1;
}

int sl_batch_create(sl_system *const *systems, int32_t k, sl_batch **out) {
    if (!out || k < 1 || !systems) return fail(SL_EINVAL, "bad arguments");
    *out = nullptr;
    if (k > sl::FUSED_MAX_SLOTS) return fail(SL_EINVAL, "at most %d slots in a batch", sl::FUSED_MAX_SLOTS);
    int prec = -1;
    for (int i = 0; i < k; ++i) {
        if (!systems[i]) continue;
        if (prec >= 0 && systems[i]->s.prec != prec) return fail(SL_EINVAL, "mixed precision modes in a batch");
        prec = systems[i]->s.prec;
        for (int j = 0; j < i; ++j)
            if (systems[j] == systems[i]) return fail(SL_EINVAL, "a system in two slots of a batch");
    }
    sl_batch *b = new (std::nothrow) sl_batch();
    if (!b) return fail(SL_ENOMEM, "host allocation failed");
    b->sys.assign(systems, systems + k);
    *out = b;
    return SL_OK;
}

int sl_batch_set(sl_batch *b, int32_t slot, sl_system *sys) {
    if (!b) return fail(SL_EINVAL, "NULL batch");
    if (slot < 0 || slot >= (int)b->sys.size()) return fail(SL_EINVAL, "slot %d outside [0, %d)", slot, (int)b->sys.size());
    for (const auto &f : b->in_flight)
        if (f.first == slot) return fail(SL_EINVAL, "slot %d takes part in a call not yet waited for", slot);
    if (sys) {
        const int prec = batch_precision(b, slot);
        if (prec >= 0 && sys->s.prec != prec) return fail(SL_EINVAL, "mixed precision modes in a batch");
        for (int i = 0; i < (int)b->sys.size(); ++i)
            if (i != slot && b->sys[i] == sys) return fail(SL_EINVAL, "the system already holds slot %d", i);
    }
    b->sys[slot] = sys;
    return SL_OK;
}

// Build (or reuse) the fork/join graph of g steps for every occupied slot.
static int batch_graph(sl_batch *b, int g) {
    const int k = (int)b->sys.size();
    // systems are told apart by id: one created after another was destroyed may reuse its address
    bool fresh = b->graph && b->graph_steps == g && (int)b->graph_uids.size() == k;
    for (int i = 0; fresh && i < k; ++i)
        fresh = b->graph_uids[i] == (b->sys[i] ? b->sys[i]->s.uid : 0) &&
                (!b->sys[i] || b->versions[i] == b->sys[i]->s.capture_version);
    if (fresh) return SL_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    CK(cudaEventRecord(b->ev[0], b->stream));
    for (int i = 0; i < k; ++i) {
        if (!b->sys[i]) continue;
        sl::Sys &s = b->sys[i]->s;
        CK(cudaStreamWaitEvent(s.stream, b->ev[0], 0));
        for (int t = 0; t < g; ++t) enqueue_step(s);
        CK(cudaEventRecord(b->ev[1 + i], s.stream));
        CK(cudaStreamWaitEvent(b->stream, b->ev[1 + i], 0));
    }
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph instantiate");
    b->graph_steps = g;
    b->graph_uids.assign((size_t)k, 0);
    b->versions.assign((size_t)k, 0);
    for (int i = 0; i < k; ++i)
        if (b->sys[i]) {
            b->graph_uids[i] = b->sys[i]->s.uid;
            b->versions[i] = b->sys[i]->s.capture_version;
        }
    return SL_OK;
}

// Whether the replicas taking part can take the fused step: one device, one model, no
// midpoint iteration.
static bool fusable(const sl_batch *b, const std::vector<int> &active) {
    if (active.empty()) return false;
    const sl::Sys &m = b->sys[active[0]]->s;
    for (int i : active) {
        const sl::Sys &s = b->sys[i]->s;
        if (s.device != m.device || s.mid_iters > 0) return false;
        if (std::memcmp(&s.pd, &m.pd, sizeof m.pd) != 0 || std::memcmp(&s.pf, &m.pf, sizeof m.pf) != 0) return false;
    }
    return true;
}

// The fused step for the replicas taking part: their budgets (n_steps) go to the device, then
// g-step graphs and one-step graphs run until the largest budget is spent.
static int fused_steps(sl_batch *b, const std::vector<int> &active, const int64_t *n_steps) {
    const int k = (int)b->sys.size();
    const sl::Sys &m = b->sys[active[0]]->s;
    sl::FusedBatch &f = b->fused;
    if (!f.ready(m.prec, k, m.device) && !f.setup(m.prec, k, m.device))
        return fail(SL_ENOMEM, "fused batch tables (%d slots)", k);
    for (int i = 0; i < k; ++i) f.assign(i, b->sys[i] ? &b->sys[i]->s : nullptr);
    f.reserve(b->reserve_atoms);
    std::vector<int64_t> left((size_t)k, 0);
    int64_t most = 0;
    for (int i : active) {
        left[(size_t)i] = n_steps[i];
        most = std::max(most, n_steps[i]);
    }
    CK(f.upload(left.data(), b->stream));   // may grow the grids, which drops the graphs
    const int g = std::max(1, m.steps_per_graph);
    if (!f.graphs(g, m, b->stream)) {
        cudaGetLastError();
        return fail(SL_ECUDA, "fused batch graph capture");
    }
    for (int i : active) {   // the batch stream waits for each replica's uploads
        sl::Sys &s = b->sys[i]->s;
        CK(cudaEventRecord(b->ev[1 + i], s.stream));
        CK(cudaStreamWaitEvent(b->stream, b->ev[1 + i], 0));
    }
    for (int64_t r = 0; r < most / g; ++r) CK(cudaGraphLaunch(f.graph_g, b->stream));
    for (int64_t r = 0; r < most % g; ++r) CK(cudaGraphLaunch(f.graph_1, b->stream));
    b->graph_launches += most / g + most % g;
    b->fused_steps += most;
    b->kernel_launches += most * sl::FUSED_LAUNCHES_PER_STEP;
    ++b->fused_calls;
    CK(cudaEventRecord(b->ev[0], b->stream));
    for (int i : active) CK(cudaStreamWaitEvent(b->sys[i]->s.stream, b->ev[0], 0));   // and each replica waits for it
    return SL_OK;
}

// Replicas on their own streams: the fork/join graph when every occupied slot takes part,
// then each replica's own graphs and single steps for the rest.
static int replica_steps(sl_batch *b, const std::vector<int> &active, const int64_t *n_steps) {
    const int k = (int)b->sys.size();
    int occupied = 0;
    for (int i = 0; i < k; ++i) occupied += b->sys[i] != nullptr;
    int rc;
    const int g = b->sys[active[0]]->s.steps_per_graph;
    bool common = g > 0 && (int)active.size() == occupied;
    int64_t shared = INT64_MAX;
    for (int i : active) {
        const sl::Sys &s = b->sys[i]->s;
        common = common && s.steps_per_graph == g && s.device == b->sys[active[0]]->s.device;
        shared = std::min<int64_t>(shared, n_steps[i]);
    }
    const int64_t rounds = common ? shared / g : 0;
    if (rounds > 0) {
        if ((rc = batch_graph(b, g))) return rc;
        for (int i : active) {   // the batch stream waits for each replica's uploads
            sl::Sys &s = b->sys[i]->s;
            CK(cudaEventRecord(b->ev[1 + i], s.stream));
            CK(cudaStreamWaitEvent(b->stream, b->ev[1 + i], 0));
        }
        for (int64_t r = 0; r < rounds; ++r) CK(cudaGraphLaunch(b->graph, b->stream));
        b->graph_launches += rounds;
        CK(cudaEventRecord(b->ev[0], b->stream));
        for (int i : active) {   // and each replica's stream waits for the batch
            sl::Sys &s = b->sys[i]->s;
            CK(cudaStreamWaitEvent(s.stream, b->ev[0], 0));
            s.n_launches += rounds * g * kernels_per_step(s);
            b->kernel_launches += rounds * g * kernels_per_step(s);
        }
    }
    for (int i : active) {
        sl::Sys &s = b->sys[i]->s;
        const int64_t left = n_steps[i] - rounds * g;
        if (left > 0) {
            if ((rc = queue_steps(s, left))) return rc;
            b->kernel_launches += left * kernels_per_step(s);
        }
    }
    ++b->replica_calls;
    return SL_OK;
}

// Queue a call's steps (fused or on the replicas' own streams) and return; the replicas taking
// part are recorded as in flight.
int sl_batch_submit(sl_batch *b, const int64_t *n_steps, const double *dt, const double *T, const double *B) {
    NvtxRange nvtx_range("sl_batch_submit");
    if (!b || !n_steps || !dt || !T || !B) return fail(SL_EINVAL, "NULL argument");
    if (!b->in_flight.empty()) return fail(SL_EINVAL, "a submitted call has not been waited for");
    const int k = (int)b->sys.size();
    for (int i = 0; i < k; ++i) {
        if (!b->sys[i]) {
            if (n_steps[i] != 0) return fail(SL_EINVAL, "steps for empty slot %d", i);
            continue;
        }
        if (b->sys[i]->s.sts) return fail(SL_EINVAL, "replica %d uses the coloured sweep, which steps alone", i);
        if (n_steps[i] < 0 || !(dt[i] > 0) || !(T[i] >= 0) || !std::isfinite(dt[i]) || !std::isfinite(T[i]))
            return fail(SL_EINVAL, "bad step arguments for replica %d", i);
    }
    int rc;
    std::vector<int> active;
    for (int i = 0; i < k; ++i) {
        if (!b->sys[i]) continue;
        sl::Sys &s = b->sys[i]->s;
        cudaSetDevice(s.device);
        if ((rc = upload_params(s, dt[i], T[i], B + 3 * i))) return rc;
        for (int c = 0; c < 3; ++c) s.B[c] = B[3 * i + c];
        if (n_steps[i] == 0 || s.n == 0) { s.step += (uint64_t)n_steps[i]; continue; }
        if ((rc = snapshot_state(s))) return rc;
        active.push_back(i);
    }
    if (active.empty()) return SL_OK;
    cudaSetDevice(b->sys[active[0]]->s.device);
    if (!b->stream) CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    if ((int)b->ev.size() != k + 1) {
        for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
        b->ev.assign((size_t)k + 1, nullptr);
        for (auto &e : b->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    rc = fusable(b, active) ? fused_steps(b, active, n_steps) : replica_steps(b, active, n_steps);
    if (rc) {   // nothing is left running for the caller to wait for
        for (int i : active) cudaStreamSynchronize(b->sys[i]->s.stream);
        if (b->stream) cudaStreamSynchronize(b->stream);
        return rc;
    }
    for (int i : active) b->in_flight.emplace_back(i, n_steps[i]);
    return SL_OK;
}

// Finish the submitted call: every replica is finished (and restored to its state before the
// call where it failed) before the first error is returned.
int sl_batch_wait(sl_batch *b) {
    NvtxRange nvtx_range("sl_batch_wait");
    if (!b) return fail(SL_EINVAL, "NULL batch");
    std::vector<std::pair<int, int64_t>> flight;
    flight.swap(b->in_flight);
    int first = SL_OK, rc;
    std::string first_msg;
    for (const auto &f : flight) {
        sl::Sys &s = b->sys[f.first]->s;
        cudaSetDevice(s.device);
        char who[32];
        std::snprintf(who, sizeof who, "replica %d: ", f.first);
        rc = finish_steps(s, f.second, who);
        if (rc && first == SL_OK) { first = rc; first_msg = g_err; }
    }
    if (first != SL_OK) return fail(first, "%s", first_msg.c_str());
    return SL_OK;
}

int sl_batch_step(sl_batch *b, const int64_t *n_steps, const double *dt, const double *T, const double *B) {
    const int rc = sl_batch_submit(b, n_steps, dt, T, B);
    if (rc) return rc;
    return sl_batch_wait(b);
}

int sl_batch_reserve(sl_batch *b, int64_t atoms) {
    if (!b || atoms < 0) return fail(SL_EINVAL, "bad arguments");
    b->reserve_atoms = std::max(b->reserve_atoms, atoms);
    return SL_OK;
}

int sl_batch_graph_launches(const sl_batch *b, int64_t *launches) {
    if (!b || !launches) return fail(SL_EINVAL, "NULL argument");
    *launches = b->graph_launches;
    return SL_OK;
}

int sl_batch_stats(const sl_batch *b, int64_t *stats) {
    if (!b || !stats) return fail(SL_EINVAL, "NULL argument");
    stats[0] = b->graph_launches;
    stats[1] = b->fused.captures;
    stats[2] = b->fused_steps;
    stats[3] = b->kernel_launches;
    stats[4] = b->fused_calls;
    stats[5] = b->replica_calls;
    stats[6] = b->fused.atom_capacity();
    return SL_OK;
}

void sl_batch_destroy(sl_batch *b) {
    if (!b) return;
    if (b->fused.device() >= 0) cudaSetDevice(b->fused.device());
    if (b->stream) cudaStreamSynchronize(b->stream);
    delete b;
}

// ---------------------------------------------------------------- no device allocation
int sl_descriptors_energies_noalloc(const double *positions4, const double *spins4, const int32_t *species,
                                    int64_t n, const double box[3], const int32_t periodic[3],
                                    const sl_nep_params *params, double *q, double *atom_energy, void *cuda_stream) {
    using namespace sl;
    if (!box || !periodic || !params) return fail(SL_EINVAL, "box, periodic and params are required");
    if (n < 0 || n > noalloc_max_atoms())
        return fail(SL_EINVAL, "n = %lld outside [0, %d], the size limit of the no-allocation scratch", (long long)n,
                    noalloc_max_atoms());
    if (n > 0 && (!positions4 || !spins4 || !species || !atom_energy))
        return fail(SL_EINVAL, "positions4, spins4, species and atom_energy are required");
    if (params->n_species != NS || params->n_ch != NCH || params->l_max != 4 || params->basis_k != NK ||
        params->n_hidden != NH || !(params->rc_ang > 0 && params->rc_rad >= params->rc_ang) || !params->coeffs ||
        !params->q_scaler || !params->w0 || !params->b0 || !params->w1)
        return fail(SL_EINVAL, "unsupported or incomplete model parameters");
    BoxDev<double> b;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0)) return fail(SL_EINVAL, "box lengths must be positive");
        if (periodic[a] && box[a] < 2.0 * params->rc_rad)
            return fail(SL_EINVAL, "periodic box length %g below 2 rc_rad", box[a]);
        b.L[a] = box[a];
        b.invL[a] = periodic[a] ? 1.0 / box[a] : 0.0;
    }
    if (n == 0) return SL_OK;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(SL_ECUDA, "no usable CUDA device");
    }
    NepDev<double> P;
    fill_params(P, params);
    int st = 0;
    if (launch_noalloc(P, reinterpret_cast<const double4 *>(positions4), reinterpret_cast<const double4 *>(spins4),
                       species, (int)n, b, q, atom_energy, (cudaStream_t)cuda_stream, &st)) {
        cudaError_t e = cudaGetLastError();
        return fail(SL_ECUDA, "no-allocation evaluation failed: %s", cudaGetErrorString(e));
    }
    if (st & ST_BAD_SPECIES) return fail(SL_EINVAL, "a species value outside [0, %d)", NS);
    if (st & ST_NBR_OVERFLOW) return fail(SL_ENBR_OVERFLOW, "more than 160 neighbours inside rc_rad");
    return SL_OK;
}

// ---------------------------------------------------------------- self checks
int sl_selftest_carrier(int32_t n_samples, double rc, double *max_rel_err_f, double *max_rel_err_df) {
    if (n_samples < 1 || !(rc > 0) || !std::isfinite(rc)) return fail(SL_EINVAL, "bad self-test arguments");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(SL_ECUDA, "no usable CUDA device");
    double out[4];
    if (sl::selftest_carrier(n_samples, rc, out)) return fail(SL_ECUDA, "carrier self-test failed to run");
    if (max_rel_err_f) *max_rel_err_f = out[0] / out[2];
    if (max_rel_err_df) *max_rel_err_df = out[1] / out[3];
    return SL_OK;
}

int sl_selftest_bounded_wait(int32_t max_polls) {
    if (max_polls < 1 || max_polls > (1 << 22)) return fail(SL_EINVAL, "max_polls must be in [1, 2^22]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(SL_ECUDA, "no usable CUDA device");
    int st = 0;
    if (sl::selftest_bounded_wait(max_polls, &st)) return fail(SL_ECUDA, "bounded-wait self-test failed to run");
    if (st & sl::ST_TIMEOUT) return fail(SL_ETIMEOUT, "a bounded device wait gave up (self-test)");
    return SL_OK;
}

int sl_selftest_harmonics(int32_t n_samples, double *max_add, double *max_grad) {
    using namespace sl;
    if (n_samples < 1) return fail(SL_EINVAL, "n_samples < 1");
    uint64_t st = 0x9E3779B97F4A7C15ULL;
    auto uni = [&]() {
        st ^= st << 13; st ^= st >> 7; st ^= st << 17;
        return (double)(st >> 11) * (1.0 / 9007199254740992.0);
    };
    auto unit = [&](double u[3]) {
        double z = 2 * uni() - 1, ph = 2 * M_PI * uni(), rr = std::sqrt(1 - z * z);
        u[0] = rr * std::cos(ph); u[1] = rr * std::sin(ph); u[2] = z;
    };
    double ea = 0, eg = 0;
    for (int t = 0; t < n_samples; ++t) {
        double u[3], v[3], pu[NLM], pv[NLM];
        unit(u); unit(v);
        harm_p(u[0], u[1], u[2], pu);
        harm_p(v[0], v[1], v[2], pv);
        const double c = u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
        const double P[5] = {1, c, 0.5 * (3 * c * c - 1), 0.5 * (5 * c * c * c - 3 * c),
                             0.125 * (35 * c * c * c * c - 30 * c * c + 3)};
        double sum[5] = {0, 0, 0, 0, 0};
        for (int lm = 0; lm < NLM; ++lm) sum[harm_l(lm)] += harm_kappa(lm) * pu[lm] * pv[lm];
        for (int l = 1; l <= 4; ++l) ea = std::max(ea, std::fabs(sum[l] - P[l]));
        // gradient: central differences of the homogeneous polynomial at a generic point
        double x[3] = {u[0] * 1.3, u[1] * 1.3, u[2] * 1.3}, g[NLM][3], p1[NLM], px[NLM];
        harm_all(x[0], x[1], x[2], p1, g);
        harm_p(x[0], x[1], x[2], px);
        for (int lm = 0; lm < NLM; ++lm) eg = std::max(eg, std::fabs(p1[lm] - px[lm]));
        const double h = 1e-6;
        for (int a = 0; a < 3; ++a) {
            double xp[3] = {x[0], x[1], x[2]}, xm[3] = {x[0], x[1], x[2]}, pp[NLM], pm[NLM];
            xp[a] += h; xm[a] -= h;
            harm_p(xp[0], xp[1], xp[2], pp);
            harm_p(xm[0], xm[1], xm[2], pm);
            for (int lm = 0; lm < NLM; ++lm) eg = std::max(eg, std::fabs((pp[lm] - pm[lm]) / (2 * h) - g[lm][a]));
        }
    }
    if (max_add) *max_add = ea;
    if (max_grad) *max_grad = eg;
    return SL_OK;
}

}  // extern "C"
