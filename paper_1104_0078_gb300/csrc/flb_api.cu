// flb_api.cu -- host runtime behind the C ABI of include/flb.h: parameter
// validation, carving of the caller's device workspace, equilibrium and state
// import/export, the per-step launch sequence and the observables.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <algorithm>
#include <cstdio>
#include <functional>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "flb_internal.cuh"
#include "flb_obs.cuh"

using namespace flb;

namespace {
// NVTX range over a scope (the calls are no-ops unless a profiler is attached):
// flb_step, and per replica step its mu, collide-stream, velocity, psi and
// sampling phases, name the launches in a trace.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

namespace flb {
// flb_lb.cu: padded plane (ghost frame of periodic images) from an interior field
cudaError_t launch_pad(const Geom &g, const float *interior, float *padded, cudaStream_t st);
cudaError_t launch_unpad(const Geom &g, const float *padded, float *interior, cudaStream_t st);
}  // namespace flb

namespace {

// ---- velocity sets in the kernels' plane order ----------------------------
const int C19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
                        {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},
                        {-1, 0, 1}, {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
const int C15[15][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                        {0, 0, 1},  {0, 0, -1}, {1, 1, 1},   {-1, -1, -1}, {1, 1, -1},
                        {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {1, -1, -1}, {-1, 1, 1}};
const int C9[9][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                      {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

inline const int *cvec(int q, int i) { return q == 19 ? C19[i] : q == 15 ? C15[i] : C9[i]; }
inline double wgt(int q, int i)
{
    const int *c = cvec(q, i);
    const int l2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    if (q == 19) return l2 == 0 ? 1.0 / 3.0 : l2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
    if (q == 15) return l2 == 0 ? 2.0 / 9.0 : l2 == 1 ? 1.0 / 9.0 : 1.0 / 72.0;
    return l2 == 0 ? 4.0 / 9.0 : l2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0;
}

// norms of the noisy modes in noise order (hand-derived from the monomials)
const double NORM19[15] = {2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 2.0 / 27, 2.0 / 27,
                           2.0 / 27, 2.0 / 9, 2.0 / 9, 2.0 / 9, 2.0 / 9, 1.0 / 3, 1.0 / 9};
// D3Q15 ghosts: c_a(c^2 - 5/3) (8/27 each), c_x c_y c_z (1/9), c^4 - 3c^2 + 4/3 (8/9)
const double NORM15[11] = {2.0 / 3, 4.0 / 3, 4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 8.0 / 27, 8.0 / 27, 8.0 / 27, 1.0 / 9, 8.0 / 9};
const double NORM9[6] = {4.0 / 9, 4.0 / 9, 1.0 / 9, 2.0 / 27, 2.0 / 27, 16.0 / 81};

constexpr long long WIN_MAX = 32768;  // sites of one flb_get_window call
constexpr int RED_MAX_BLOCKS = 1024;

struct Rep {
    flb_params p;
    Geom g;
    int q = 0, dim = 0;
    size_t pop_elem = 4;
    void *f[2] = {nullptr, nullptr};
    int cur = 0;
    float *psi[2] = {nullptr, nullptr};
    int pcur = 0;
    float *psis = nullptr, *mu = nullptr, *mus = nullptr, *u = nullptr, *J = nullptr, *eta = nullptr, *E = nullptr;
    float *sig = nullptr;  // stress-form force: sigma planes (3D xx, yy, zz, xy, xz, yz; 2D xx, yy, xy)
    float *Dn = nullptr;   // RK4 (3D): the step's noise increment per site
    double *sq = nullptr, *hsq = nullptr;
    int Kx = 0, Ky = 0, Kz = 0;
    int64_t sq_n = 0, h_n = 0;
    float2 *dring = nullptr;   // dynamic S(q, tau): last sq_lags Fourier snapshots
    double *dacc = nullptr;    // and the lag accumulators, sq_lags x K
    int dslot = -1;
    int64_t d_n = 0;
    int64_t step = 0;
    float omega_s = 0, omega_b = 0, gamma_g = 0;
    float namp[16] = {0};
    int zc = PS_ZC;  // planes per psi block (3D), set by flb_set_tuning / flb_autotune
    int fused = 0;   // single-pass Heun psi step (flb_set_psi_fused)
};

struct Carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

int axis_K(int n, int kmax) { return (kmax <= 0 || 2 * kmax + 1 >= n) ? n : 2 * kmax + 1; }

bool valid(const flb_params &p)
{
    if (!((p.dim == 3 && (p.q == 19 || p.q == 15)) || (p.dim == 2 && p.q == 9))) return false;
    if (p.laplacian < FLB_LAP_SO || p.laplacian > (p.dim == 3 ? FLB_LAP_LB : FLB_LAP_CD)) return false;
    // the stress kernels evaluate lap psi with the SO stencil
    if (p.force_grad == FLB_FORCE_STRESS && p.laplacian != FLB_LAP_SO) return false;
    const long long nz = p.dim == 3 ? p.nz : 1;
    if (p.nx < 4 || p.ny < 4 || (p.dim == 3 && p.nz < 4)) return false;
    if (p.init < FLB_INIT_REST || p.init > FLB_INIT_USER) return false;
    // the equilibrium start draws psi from the Gaussian law kT/(A - K L(q))
    if (p.init == FLB_INIT_EQUILIBRIUM && !(p.A > 0 && p.K >= 0 && p.kT >= 0)) return false;
    if ((long long)p.nx * p.ny * nz >= (1LL << 31)) return false;
    if ((long long)(p.nx + 2 * GX + 3) * (p.ny + 2 * GY) * (nz + (p.dim == 3 ? 2 * GZ3 : 0)) >= (1LL << 31)) return false;
    if (!(p.rho0 > 0) || !(p.tau > 0) || !std::isfinite(p.tau) || !std::isfinite(p.rho0)) return false;
    if (!std::isnan(p.gamma_bulk) && !(std::fabs(p.gamma_bulk) < 1.0)) return false;
    if (!(std::fabs(p.gamma_ghost) < 1.0)) return false;
    if (!(p.kT >= 0) || !(p.M >= 0) || !std::isfinite(p.kT) || !std::isfinite(p.M)) return false;
    if (!std::isfinite(p.A) || !std::isfinite(p.B) || !std::isfinite(p.K)) return false;
    if (p.psi_scheme != FLB_FD && p.psi_scheme != FLB_FV && p.psi_scheme != FLB_NAIVE) return false;
    if (p.integrator != FLB_EULER && p.integrator != FLB_HEUN && p.integrator != FLB_RK4) return false;
    if (p.storage != FLB_F32_DEV && p.storage != FLB_F16_DEV) return false;
    if (p.coupling < 0 || p.coupling > 3) return false;
    if (p.force_grad < FLB_FORCE_MATCHED || p.force_grad > FLB_FORCE_STRESS) return false;
    if (p.sq_kmax < 0) return false;
    if (p.sq_lags < 0 || p.sq_lags > 4096) return false;
    if (p.nx > 4096 || p.ny > 4096 || (p.dim == 3 && p.nz > 4096)) return false;  // DFT twiddle tables
    return true;
}

// 3D combinations outside the tiled kernels (another Laplacian, the naive
// scheme) run the one-thread-per-site kernels of the 2D path.
bool general_path(const flb_params &p)
{
    // the tiled 3D kernels take the FD scheme with any Laplacian (class weights)
    // and the FV scheme with the SO Laplacian
    return p.dim == 3 && (p.psi_scheme == FLB_NAIVE || (p.laplacian != FLB_LAP_SO && p.psi_scheme != FLB_FD));
}

// Class weights of the App. A Laplacians (faces, edges, corners; 2D axes and
// diagonals), the centre weight closing the sum to zero.
LapW lap_weights(int dim, int kind)
{
    LapW w{0.f, 0.f, 0.f, 0.f};
    double a1, a2, a3 = 0.0, a0;
    if (dim == 3) {
        switch (kind) {
        case FLB_LAP_CD: a1 = 1.0; a2 = 0.0; a3 = 0.0; break;
        case FLB_LAP_PK: a1 = 14.0 / 30.0; a2 = 3.0 / 30.0; a3 = 1.0 / 30.0; break;
        case FLB_LAP_LB: a1 = 1.0 / 9.0; a2 = 1.0 / 9.0; a3 = 1.0 / 9.0; break;
        default: a1 = 6.0 / 22.0; a2 = 3.0 / 22.0; a3 = 1.0 / 22.0; break;
        }
        a0 = -(6.0 * a1 + 12.0 * a2 + 8.0 * a3);
    } else {
        if (kind == FLB_LAP_CD) { a1 = 1.0; a2 = 0.0; }
        else { a1 = 0.5; a2 = 0.25; }
        a0 = -(4.0 * a1 + 4.0 * a2);
    }
    w.c0 = (float)a0;
    w.c1 = (float)a1;
    w.c2 = (float)a2;
    w.c3 = (float)a3;
    return w;
}

// The class weights of a 3D replica's App. A Laplacian on the tiled FD path
// (stored in w), or null for the SO Laplacian of the tiled kernels.
const LapW *app_a_weights(const Rep &r, LapW &w)
{
    if (r.dim != 3 || r.p.laplacian == FLB_LAP_SO || r.p.psi_scheme != FLB_FD) return nullptr;
    w = lap_weights(3, r.p.laplacian);
    return &w;
}

Geom make_geom(const flb_params &p)
{
    Geom g;
    g.dim = p.dim;
    g.nx = p.nx;
    g.ny = p.ny;
    g.nz = p.dim == 3 ? p.nz : 1;
    g.gz = p.dim == 3 ? GZ3 : 0;
    g.px = ((g.nx + 2 * GX + 3) / 4) * 4;  // row pitch a multiple of 16 bytes (TMA)
    g.py = g.ny + 2 * GY;
    g.pz = g.nz + 2 * g.gz;
    g.n = (long long)g.nx * g.ny * g.nz;
    g.pn = (long long)g.px * g.py * g.pz;
    return g;
}

// Assign the replica's device arrays from the carver (base may be null for sizing).
void carve_rep(Rep &r, Carver &cv)
{
    const Geom &g = r.g;
    const size_t N = (size_t)g.n, P = (size_t)g.pn;
    r.f[0] = cv.take<char>((size_t)r.q * N * r.pop_elem);
    r.f[1] = cv.take<char>((size_t)r.q * N * r.pop_elem);
    r.psi[0] = cv.take<float>(P);
    r.psi[1] = cv.take<float>(P);
    r.mu = cv.take<float>(P);
    r.u = cv.take<float>((size_t)r.dim * P);
    if (r.p.integrator == FLB_HEUN || r.p.integrator == FLB_RK4) {
        r.psis = cv.take<float>(P);
        r.E = cv.take<float>(N);
    }
    if (r.p.integrator == FLB_RK4 && r.dim == 3) r.Dn = cv.take<float>(N);
    if (r.dim == 2 || general_path(r.p)) {  // the per-site path keeps mu*, the noise increment and the FV flux in HBM
        r.eta = cv.take<float>(N);
        if (r.p.integrator != FLB_EULER) r.mus = cv.take<float>(P);
        if (r.p.psi_scheme == FLB_FV) r.J = cv.take<float>((size_t)r.dim * P);
    }
    if (r.p.force_grad == FLB_FORCE_STRESS) r.sig = cv.take<float>((size_t)(r.dim == 3 ? 6 : 3) * P);
    r.Kx = axis_K(g.nx, r.p.sq_kmax);
    r.Ky = axis_K(g.ny, r.p.sq_kmax);
    r.Kz = r.dim == 3 ? axis_K(g.nz, r.p.sq_kmax) : 1;
    r.sq = cv.take<double>((size_t)r.Kx * r.Ky * r.Kz);
    if (r.dim == 3) r.hsq = cv.take<double>((size_t)g.nx * g.ny);
    if (r.p.sq_lags > 0) {
        const size_t K = (size_t)r.Kx * r.Ky * r.Kz;
        r.dring = cv.take<float2>(K * (size_t)r.p.sq_lags);
        r.dacc = cv.take<double>(K * (size_t)r.p.sq_lags);
    }
}

void init_rep_consts(Rep &r, const flb_params &p)
{
    r.p = p;
    r.q = p.q;
    r.dim = p.dim;
    r.g = make_geom(p);
    r.pop_elem = p.storage == FLB_F16_DEV ? 2 : 4;
    const double ws = 1.0 / (p.tau + 0.5);
    const double gs = 1.0 - ws;
    const double gb = std::isnan(p.gamma_bulk) ? gs : p.gamma_bulk;
    r.omega_s = (float)ws;
    r.omega_b = (float)(1.0 - gb);
    r.gamma_g = (float)p.gamma_ghost;
    const int nn = p.q - p.dim - 1;
    const int nstress = p.dim == 3 ? 6 : 3;
    for (int t = 0; t < nn; ++t) {
        const double gam = t == 0 ? gb : (t < nstress ? gs : p.gamma_ghost);
        const double b = p.q == 19 ? NORM19[t] : p.q == 15 ? NORM15[t] : NORM9[t];
        r.namp[t] = (float)std::sqrt((1.0 - gam * gam) / b);
    }
}

}  // namespace

struct flb_handle {
    std::vector<Rep> reps;
    cudaStream_t st = nullptr;
    int mode = FLB_MODE_PLAIN;
    int sample_every = 0, sample_mask = 0;
    int64_t launches = 0;
    double *red_partial = nullptr, *red_out = nullptr;
    int *status = nullptr;  // device status word: kernels latch FLB_ETIMEOUT here
    // batched mode: descriptor table, block lists, device step counter, captured graph
    BatchRep *b_reps = nullptr;
    BatchBlock *b_mu = nullptr, *b_lb = nullptr, *b_psi = nullptr;
    int b_nmu = 0, b_nlb = 0, b_npsi = 0, b_npsi_cap = 0;
    long long *b_dstep = nullptr;
    std::vector<BatchRep> b_host;
    std::vector<BatchBlock> b_blocks_host;
    cudaGraph_t b_graph = nullptr;
    cudaGraphExec_t b_exec = nullptr;
    bool b_lists_ok = false;
    // persistent mode: one step's task list, dispatch and completion counters
    PTask *p_tasks = nullptr;
    size_t p_cap = 0;
    int p_ntask = 0;
    unsigned *p_ticket = nullptr, *p_done = nullptr;
    int *p_abort = nullptr;
    std::vector<int> p_pstep;
    bool p_ok = false;
    unsigned long long wait_ns = 1000000000ull;  // 1 s per inter-block wait
    float2 *X1 = nullptr, *X2 = nullptr;
    float *heights = nullptr, *win = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    // per-phase timing (flb_set_profiling)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[3];
    int64_t phase_launches[3] = {0, 0, 0};
    // host staging of the FP32 fields that set_fields and get_psi_u move; kept
    // between calls (grown, never shrunk) so that a call neither clears nor
    // first-touches a fresh buffer
    std::vector<float> hstage;
    float *host_stage(size_t n)
    {
        if (hstage.size() < n) hstage.resize(n);
        return hstage.data();
    }
    ~flb_handle()
    {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        if (b_exec) cudaGraphExecDestroy(b_exec);
        if (b_graph) cudaGraphDestroy(b_graph);
    }
};

namespace {

size_t carve_all(flb_handle &h, char *base)
{
    Carver cv{base};
    size_t cap1 = 0, cap2 = 0, hcap = 0;
    long long maxq = 0;
    for (Rep &r : h.reps) {
        carve_rep(r, cv);
        const Geom &g = r.g;
        cap1 = std::max(cap1, (size_t)g.nz * g.ny * r.Kx);
        cap2 = std::max(cap2, (size_t)g.nz * r.Ky * r.Kx);
        if (r.dim == 3) {
            cap1 = std::max(cap1, (size_t)g.ny * g.nx);
            cap2 = std::max(cap2, (size_t)g.ny * g.nx);
            hcap = std::max(hcap, (size_t)2 * g.nx * g.ny);
        }
        maxq = std::max<long long>(maxq, r.q);
    }
    // batched-mode block lists (3D replicas only)
    int nmu = 0, nlb = 0, npsi = 0;
    for (Rep &r : h.reps) {
        if (r.dim != 3) continue;
        const Geom &g = r.g;
        constexpr int E = 2 * MU3_HALO;
        nmu += ((g.nx + E + MU_BX - 1) / MU_BX) * ((g.ny + E + MU_BY - 1) / MU_BY) * ((g.nz + E + MU_ZC - 1) / MU_ZC);
        nlb += packed_blocks(pair_geom(g), LBB_NT);
        npsi += ((g.nx + PS_TX - 1) / PS_TX) * ((g.ny + PS_TY - 1) / PS_TY) * ((g.nz + PS_ZC_MIN - 1) / PS_ZC_MIN);
    }
    h.b_nmu = nmu;
    h.b_nlb = nlb;
    h.b_npsi = npsi;
    h.b_npsi_cap = npsi;
    h.b_reps = cv.take<BatchRep>(h.reps.size());
    h.b_mu = cv.take<BatchBlock>((size_t)std::max(nmu, 1));
    h.b_lb = cv.take<BatchBlock>((size_t)std::max(nlb, 1));
    h.b_psi = cv.take<BatchBlock>((size_t)std::max(npsi, 1));
    h.b_dstep = cv.take<long long>(1);
    // persistent-mode task list, sized for the smallest psi depth
    size_t ptask = 0;
    for (Rep &r : h.reps) {
        if (r.dim != 3) continue;
        int c[PH_COUNT];
        persist_tiles(r.g, PS_ZC_MIN, FLB_COUPLE_FORCE, 1, c);
        for (int k = 0; k < PH_COUNT; ++k) ptask += (size_t)c[k];
    }
    h.p_cap = ptask;
    h.p_tasks = cv.take<PTask>(std::max<size_t>(ptask, 1));
    h.p_ticket = cv.take<unsigned>(1);
    h.p_abort = cv.take<int>(1);
    h.p_done = cv.take<unsigned>(h.reps.size());
    h.red_partial = cv.take<double>((size_t)RED_MAX_BLOCKS * std::max(NRED, NMSQ));
    h.red_out = cv.take<double>(std::max(NRED, NMSQ));
    h.status = cv.take<int>(1);
    h.X1 = cv.take<float2>(cap1);
    h.X2 = cv.take<float2>(cap2);
    h.heights = cv.take<float>(std::max<size_t>(hcap, 1));
    h.win = cv.take<float>((size_t)WIN_MAX * (maxq + 1));
    return cv.off + 256;
}

int cuerr(cudaError_t e) { return e == cudaSuccess ? FLB_OK : FLB_ECUDA; }

// Record a timing event on the handle's stream (no-op unless profiling).
cudaEvent_t mark(flb_handle *h)
{
    if (!h->profiling) return nullptr;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    cudaEvent_t e = h->ev_pool[h->ev_used++];
    cudaEventRecord(e, h->st);
    return e;
}

void span(flb_handle *h, int phase, cudaEvent_t a, cudaEvent_t b, int launches)
{
    if (!h->profiling || !a || !b) return;
    h->spans[phase].push_back({a, b});
    h->phase_launches[phase] += launches;
}

// physical fbar (FP64, [q][N]) -> stored post-collision deviations at origin sites
void phys_to_stored(const Rep &r, const double *f, std::vector<float> &out)
{
    const Geom &g = r.g;
    const long long N = g.n;
    out.resize((size_t)r.q * N);
    for (int i = 0; i < r.q; ++i) {
        const int *c = cvec(r.q, i);
        const double wr = wgt(r.q, i) * r.p.rho0;
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < g.ny; ++y)
                for (int x = 0; x < g.nx; ++x) {
                    // stored_i(y) = fbar_i(y + c_i)
                    const long long src = g.sidx(wrapi(x + c[0], g.nx), wrapi(y + c[1], g.ny),
                                                 g.dim == 3 ? wrapi(z + c[2], g.nz) : 0);
                    out[(size_t)i * N + g.sidx(x, y, z)] = (float)(f[(size_t)i * N + src] - wr);
                }
    }
}

int upload_pops(flb_handle *h, Rep &r, const std::vector<float> &dev)
{
    const size_t n = dev.size();
    if (r.pop_elem == 4) return cuerr(cudaMemcpyAsync(r.f[r.cur], dev.data(), n * 4, cudaMemcpyHostToDevice, h->st));
    std::vector<__half> hv(n);
    for (size_t k = 0; k < n; ++k) hv[k] = __float2half_rn(dev[k]);
    int rc = cuerr(cudaMemcpyAsync(r.f[r.cur], hv.data(), n * 2, cudaMemcpyHostToDevice, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    return rc;
}

int download_pops(flb_handle *h, Rep &r, std::vector<float> &dev)
{
    const size_t n = (size_t)r.q * r.g.n;
    dev.resize(n);
    if (r.pop_elem == 4) {
        int rc = cuerr(cudaMemcpyAsync(dev.data(), r.f[r.cur], n * 4, cudaMemcpyDeviceToHost, h->st));
        return rc == FLB_OK ? cuerr(cudaStreamSynchronize(h->st)) : rc;
    }
    std::vector<__half> hv(n);
    int rc = cuerr(cudaMemcpyAsync(hv.data(), r.f[r.cur], n * 2, cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    for (size_t k = 0; k < n; ++k) dev[k] = __half2float(hv[k]);
    return rc;
}

// interior values (FP32, [N]) -> padded plane with every ghost cell filled periodically
void to_padded(const Geom &g, const float *in, std::vector<float> &out)
{
    out.assign((size_t)g.pn, 0.f);
    for (int z = -g.gz; z < g.nz + g.gz; ++z)
        for (int y = -GY; y < g.ny + GY; ++y)
            for (int x = -GX; x < g.nx + GX; ++x)
                out[(size_t)g.pidx(x, y, z)] =
                    in[g.sidx(((x % g.nx) + g.nx) % g.nx, ((y % g.ny) + g.ny) % g.ny, ((z % g.nz) + g.nz) % g.nz)];
}

int upload_padded(flb_handle *h, const Geom &g, float *dst, const float *interior)
{
    std::vector<float> pad;
    to_padded(g, interior, pad);
    int rc = cuerr(cudaMemcpyAsync(dst, pad.data(), pad.size() * 4, cudaMemcpyHostToDevice, h->st));
    return rc == FLB_OK ? cuerr(cudaStreamSynchronize(h->st)) : rc;
}

int download_interior(flb_handle *h, const Geom &g, const float *src, std::vector<float> &out)
{
    std::vector<float> pad((size_t)g.pn);
    int rc = cuerr(cudaMemcpyAsync(pad.data(), src, pad.size() * 4, cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    out.resize((size_t)g.n);
    for (int z = 0; z < g.nz; ++z)
        for (int y = 0; y < g.ny; ++y)
            for (int x = 0; x < g.nx; ++x) out[(size_t)g.sidx(x, y, z)] = pad[(size_t)g.pidx(x, y, z)];
    return rc;
}

#define FLB_TRY(expr)                     \
    do {                                  \
        const cudaError_t e_ = (expr);    \
        ++h->launches;                    \
        if (e_ != cudaSuccess) return FLB_ECUDA; \
    } while (0)

// One coupled step of one replica: LB (reads psi^n, mu^n; writes u^n), then psi.
LBArgs lb_args(const Rep &r, float *psi_n)
{
    const flb_params &p = r.p;
    LBArgs la;
    la.g = r.g;
    la.fin = r.f[r.cur];
    la.fout = r.f[r.cur ^ 1];
    la.psi = psi_n;
    la.mu = r.mu;
    la.u = r.u;
    la.rho0 = (float)p.rho0;
    la.omega_s = r.omega_s;
    la.omega_b = r.omega_b;
    la.gamma_g = r.gamma_g;
    la.kT = (float)p.kT;
    std::memcpy(la.namp, r.namp, sizeof(la.namp));
    {
        const double ws = r.omega_s, wb = r.omega_b, cs = 1.0 - 0.5 * ws, cb = 1.0 - 0.5 * wb;
        la.rq[0] = (float)(4.5 * (1.0 - ws));
        la.rq[1] = (float)(4.5 * ws);
        la.rq[2] = (float)(4.5 * cs);
        la.rq[3] = (float)(1.5 * (wb - ws));
        la.rq[4] = (float)(3.0 * (cb - cs));
        la.iso = r.omega_s != r.omega_b;
        la.k3T = (float)(3.0 * p.kT);
        // Q = 4.5 B takes the stress noise at 4.5 x (2/9, 1/9); the ghosts G10-G12,
        // G16 are g/3 and G17, G18 are g/2
        const double sc[15] = {1, 1, 1, 0.5, 0.5, 0.5, 1.0 / 3, 1.0 / 3, 1.0 / 3, 1, 1, 1, 1.0 / 3, 0.5, 0.5};
        for (int t = 0; t < 15; ++t) la.nq[t] = (float)(sc[t] * (double)r.namp[t]);
    }
    la.coupling = p.coupling;
    const bool fv_grad =
        p.force_grad == FLB_FORCE_FV || (p.force_grad == FLB_FORCE_MATCHED && p.psi_scheme == FLB_FV);
    la.force_kind = p.force_grad == FLB_FORCE_STRESS ? 2 : fv_grad ? (p.q == 15 ? 3 : 1) : 0;
    la.sig = r.sig;
    la.key = philox_key(p.seed);
    la.step = r.step;
    return la;
}

// The Runge-Kutta stages of psi (3D) for the current step of replica r, advected
// by the velocity in r.u.  They write only step scratch (psi*, E) and the other
// psi buffer, so repeating them leaves the state unchanged (the autotuner relies
// on it).  Stage 1 takes mu of psi^n from r.mu when the step formed it there for
// the force (FV stage 1 then skips forming it).
int launch_psi_stages(flb_handle *h, Rep &r)
{
    const flb_params &p = r.p;
    cudaStream_t st = h->st;
    LapW lwv{};
    const LapW *lw = app_a_weights(r, lwv);
    float *psi_n = r.psi[r.pcur], *psi_np1 = r.psi[r.pcur ^ 1];
    const float *mu_n = (p.coupling & FLB_COUPLE_FORCE) && p.force_grad != FLB_FORCE_STRESS ? r.mu : nullptr;
    const bool noisy = p.kT > 0 && p.M > 0;
    const bool heun = p.integrator == FLB_HEUN;
    const int advect = (p.coupling & FLB_COUPLE_ADVECT) ? 1 : 0;
    const PhiloxKey key = philox_key(p.seed);
    if (p.integrator == FLB_RK4) {
        // stage inputs and outputs alternate between psi* and the spare psi buffer
        const float *in[4] = {psi_n, r.psis, psi_np1, r.psis};
        float *out[4] = {r.psis, psi_np1, r.psis, psi_np1};
        for (int s = 0; s < 4; ++s)
            FLB_TRY(launch_psi3(r.g, p.psi_scheme, r.q, s == 0 ? 1 : 2, s == 0 && noisy, in[s], r.u, out[s], r.E,
                                (float)p.A, (float)p.B, (float)p.K, (float)p.M, (float)p.kT, advect, 0, key, r.step,
                                r.zc, s + 1, psi_n, r.Dn, s == 0 ? mu_n : nullptr, h->status, st, lw));
        return FLB_OK;
    }
    if (r.fused && heun) {  // both stages in one launch (flb_set_psi_fused)
        FLB_TRY(launch_psi3_heun1(r.g, p.psi_scheme, psi_n, r.u, psi_np1, (float)p.A, (float)p.B, (float)p.K,
                                  (float)p.M, (float)p.kT, advect, noisy, key, r.step, r.zc, st));
        return FLB_OK;
    }
    FLB_TRY(launch_psi3(r.g, p.psi_scheme, r.q, 1, noisy, psi_n, r.u, heun ? r.psis : psi_np1, r.E, (float)p.A,
                        (float)p.B, (float)p.K, (float)p.M, (float)p.kT, advect, heun ? 1 : 0, key, r.step, r.zc, 0,
                        nullptr, nullptr, mu_n, h->status, st, lw));
    if (heun)
        FLB_TRY(launch_psi3(r.g, p.psi_scheme, r.q, 2, false, r.psis, r.u, psi_np1, r.E, (float)p.A, (float)p.B,
                            (float)p.K, (float)p.M, (float)p.kT, advect, 1, key, r.step, r.zc, 0, nullptr, nullptr,
                            nullptr, h->status, st, lw));
    return FLB_OK;
}

// 3D step: mu of psi^n, the collide-stream with the force -psi grad mu, the
// velocity of the new fluid state, then one fused launch per Runge-Kutta stage
// of psi advected by that velocity (Gauss-Seidel coupling).
int step_rep3(flb_handle *h, Rep &r)
{
    const flb_params &p = r.p;
    cudaStream_t st = h->st;
    float *psi_n = r.psi[r.pcur];
    const LBArgs la = lb_args(r, psi_n);
    cudaEvent_t e0 = mark(h);
    if (p.coupling & FLB_COUPLE_FORCE) {
        const Range range("mu");
        if (p.force_grad == FLB_FORCE_STRESS)
            FLB_TRY(launch_sigma3(r.g, psi_n, r.sig, (float)p.A, (float)p.B, (float)p.K, st));
        else {
            LapW lwv{};
            FLB_TRY(launch_mu3(r.g, psi_n, r.mu, (float)p.A, (float)p.B, (float)p.K, st, app_a_weights(r, lwv)));
        }
    }
    cudaEvent_t e1 = mark(h);
    {
        const Range range("collide-stream");
        FLB_TRY(r.q == 15 ? launch_lb15(la, p.storage, st) : launch_lb3d(la, p.storage, st));
    }
    cudaEvent_t e2 = mark(h);
    const int64_t l2 = h->launches;
    {
        const Range range("velocity");
        FLB_TRY(r.q == 15 ? launch_vel15(la, p.storage, st) : launch_vel3(la, p.storage, st));
    }
    int rc;
    {
        const Range range("psi");
        rc = launch_psi_stages(h, r);
    }
    if (rc != FLB_OK) return rc;
    cudaEvent_t e3 = mark(h);
    span(h, 0, e1, e2, 1);
    span(h, 1, e0, e1, (p.coupling & FLB_COUPLE_FORCE) ? 1 : 0);
    span(h, 1, e2, e3, (int)(h->launches - l2));
    r.cur ^= 1;
    r.pcur ^= 1;
    r.step += 1;
    return FLB_OK;
}

int step_rep(flb_handle *h, Rep &r)
{
    if (r.dim == 3 && !general_path(r.p)) return step_rep3(h, r);
    const Range range("step (per-site kernels)");
    // one-thread-per-site path: 2D, and the 3D combinations of general_path()
    const Geom &g = r.g;
    const flb_params &p = r.p;
    cudaStream_t st = h->st;
    const LapW lw = lap_weights(r.dim, p.laplacian);
    float *psi_n = r.psi[r.pcur], *psi_np1 = r.psi[r.pcur ^ 1];
    const int64_t l0 = h->launches;
    cudaEvent_t e0 = mark(h);
    FLB_TRY(launch_mu(g, psi_n, r.mu, (float)p.A, (float)p.B, (float)p.K, lw, st));
    if ((p.coupling & FLB_COUPLE_FORCE) && p.force_grad == FLB_FORCE_STRESS) {
        if (r.dim == 3) FLB_TRY(launch_sigma3(g, psi_n, r.sig, (float)p.A, (float)p.B, (float)p.K, st));
        else FLB_TRY(launch_sigma2(g, psi_n, r.sig, (float)p.A, (float)p.B, (float)p.K, st));
    }
    cudaEvent_t e1 = mark(h);

    const LBArgs la = lb_args(r, psi_n);
    if (r.dim == 3) FLB_TRY(r.q == 15 ? launch_lb15(la, p.storage, st) : launch_lb3d(la, p.storage, st));
    else FLB_TRY(launch_lb(la, r.q, p.storage, st));
    cudaEvent_t e2 = mark(h);
    const int64_t l2 = h->launches;
    if (r.dim == 3) FLB_TRY(r.q == 15 ? launch_vel15(la, p.storage, st) : launch_vel3(la, p.storage, st));
    else FLB_TRY(launch_vel2(la, p.storage, st));

    const bool noisy = p.kT > 0 && p.M > 0;
    if (noisy) {
        NoiseArgs na;
        na.g = g;
        na.eta = r.eta;
        na.kT = (float)p.kT;
        na.M = (float)p.M;
        na.scheme = p.psi_scheme;
        na.q = r.q;
        na.lw = lw;
        na.key = philox_key(p.seed);
        na.step = r.step;
        FLB_TRY(launch_noise(na, st));
    }
    if (p.psi_scheme == FLB_FV) FLB_TRY(launch_flux(g, r.q, psi_n, r.mu, r.u, r.J, (float)p.M, p.coupling, st));
    PsiArgs pa;
    pa.g = g;
    pa.lw = lw;
    pa.q = r.q;
    pa.psi = psi_n;
    pa.mu = r.mu;
    pa.u = r.u;
    pa.J = r.J;
    pa.eta = noisy ? r.eta : nullptr;
    pa.psi0 = nullptr;
    pa.out = p.integrator == FLB_EULER ? psi_np1 : r.psis;
    pa.acc = r.E;
    pa.base = psi_n;
    pa.A = (float)p.A;
    pa.B = (float)p.B;
    pa.K = (float)p.K;
    pa.M = (float)p.M;
    pa.coupling = p.coupling;
    pa.scheme = p.psi_scheme;
    pa.stage = 1;
    pa.integrator = p.integrator;
    FLB_TRY(launch_psi_update(pa, r.q, st));
    if (p.integrator == FLB_RK4) {  // stages 2-4 alternate between psi* and the spare psi buffer
        float *in[3] = {r.psis, psi_np1, r.psis};
        float *out[3] = {psi_np1, r.psis, psi_np1};
        for (int s = 0; s < 3; ++s) {
            FLB_TRY(launch_mu(g, in[s], r.mus, (float)p.A, (float)p.B, (float)p.K, lw, st));
            if (p.psi_scheme == FLB_FV)
                FLB_TRY(launch_flux(g, r.q, in[s], r.mus, r.u, r.J, (float)p.M, p.coupling, st));
            pa.psi = in[s];
            pa.mu = r.mus;
            pa.out = out[s];
            pa.stage = s + 2;
            FLB_TRY(launch_psi_update(pa, r.q, st));
        }
    }
    if (p.integrator == FLB_HEUN) {
        FLB_TRY(launch_mu(g, r.psis, r.mus, (float)p.A, (float)p.B, (float)p.K, lw, st));
        if (p.psi_scheme == FLB_FV)
            FLB_TRY(launch_flux(g, r.q, r.psis, r.mus, r.u, r.J, (float)p.M, p.coupling, st));
        pa.psi = r.psis;
        pa.mu = r.mus;
        pa.psi0 = r.E;
        pa.out = psi_np1;
        pa.stage = 2;
        FLB_TRY(launch_psi_update(pa, r.q, st));
    }
    cudaEvent_t e3 = mark(h);
    span(h, 0, e1, e2, 1);
    span(h, 1, e0, e1, 1);
    span(h, 1, e2, e3, (int)(h->launches - l2));
    (void)l0;
    r.cur ^= 1;
    r.pcur ^= 1;
    r.step += 1;
    return FLB_OK;
}

int sample_rep(flb_handle *h, Rep &r, int mask)
{
    const Range range("sample");
    const Geom &g = r.g;
    cudaEvent_t e0 = mark(h);
    const int64_t l0 = h->launches;
    struct Close {
        flb_handle *h;
        cudaEvent_t e0;
        int64_t l0;
        ~Close() { span(h, 2, e0, mark(h), (int)(h->launches - l0)); }
    } close_{h, e0, l0};
    const bool dyn = (mask & 4) && r.dring;
    if ((mask & 1) || dyn) {
        DftArgs d;
        d.in = r.psi[r.pcur];
        d.off = g.pidx(0, 0, 0);
        d.sy = g.px;
        d.sz = (long long)g.px * g.py;
        d.nx = g.nx;
        d.ny = g.ny;
        d.nz = g.nz;
        d.Kx = r.Kx;
        d.Ky = r.Ky;
        d.Kz = r.Kz;
        d.X1 = h->X1;
        d.X2 = h->X2;
        d.S = (mask & 1) ? r.sq : nullptr;
        d.scale = 1.0 / (double)g.n;
        const long long K = (long long)r.Kx * r.Ky * r.Kz;
        const int L = r.p.sq_lags;
        const int slot = dyn ? (r.dslot + 1) % L : 0;
        d.snap = dyn ? r.dring + (size_t)slot * K : nullptr;
        const cudaError_t e = launch_dft_accumulate(d, h->st);
        h->launches += 3;
        if (e != cudaSuccess) return FLB_ECUDA;
        if (mask & 1) r.sq_n += 1;
        if (dyn) {
            const int nlag = (int)std::min<int64_t>(r.d_n + 1, L);
            FLB_TRY(launch_dyn_corr(r.dring, L, slot, nlag, K, r.dacc, 1.0 / (double)g.n, h->st));
            r.dslot = slot;
            r.d_n += 1;
        }
    }
    if ((mask & 2) && r.dim == 3) {
        FLB_TRY(launch_heights(g, r.psi[r.pcur], h->heights, h->st));
        for (int part = 0; part < 2; ++part) {
            DftArgs d;
            d.in = h->heights;
            d.off = (long long)part * g.nx * g.ny;
            d.sy = g.nx;
            d.sz = 0;
            d.nx = g.nx;
            d.ny = g.ny;
            d.nz = 1;
            d.Kx = g.nx;
            d.Ky = g.ny;
            d.Kz = 1;
            d.X1 = h->X1;
            d.X2 = h->X2;
            d.S = r.hsq;
            d.scale = 0.5 / ((double)g.nx * g.ny);
            const cudaError_t e = launch_dft_accumulate(d, h->st);
            h->launches += 3;
            if (e != cudaSuccess) return FLB_ECUDA;
        }
        r.h_n += 1;
    }
    return FLB_OK;
}

// Read and clear the device status word (after the stream has drained).
int take_status(flb_handle *h)
{
    int s = 0;
    if (cudaMemcpyAsync(&s, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->st) != cudaSuccess) return FLB_ECUDA;
    if (cudaStreamSynchronize(h->st) != cudaSuccess) return FLB_ECUDA;
    if (s != 0 && cudaMemsetAsync(h->status, 0, sizeof(int), h->st) != cudaSuccess) return FLB_ECUDA;
    return s;
}

// ---- batched mode ---------------------------------------------------------
bool batch_supported(const flb_handle *h)
{
    for (const Rep &r : h->reps)
        if (r.dim != 3 || r.p.psi_scheme != FLB_FV || r.p.integrator == FLB_RK4 || r.p.laplacian != FLB_LAP_SO)
            return false;
    return !h->reps.empty();
}

int batch_upload_lists(flb_handle *h)
{
    std::vector<BatchBlock> &v = h->b_blocks_host;
    v.clear();
    for (int r = 0; r < (int)h->reps.size(); ++r) {
        const Geom &g = h->reps[(size_t)r].g;
        constexpr int E = 2 * MU3_HALO;
        for (int bz = 0; bz < (g.nz + E + MU_ZC - 1) / MU_ZC; ++bz)
            for (int by = 0; by < (g.ny + E + MU_BY - 1) / MU_BY; ++by)
                for (int bx = 0; bx < (g.nx + E + MU_BX - 1) / MU_BX; ++bx) v.push_back({r, bx, by, bz});
    }
    const size_t nmu = v.size();
    for (int r = 0; r < (int)h->reps.size(); ++r)  // row-packed collide-stream / velocity blocks
        for_packed_blocks(pair_geom(h->reps[(size_t)r].g), LBB_NT,
                          [&](int x0, int y0, int z0) { v.push_back({r, x0, y0, z0}); });
    const size_t nlb = v.size() - nmu;
    for (int r = 0; r < (int)h->reps.size(); ++r) {
        const Geom &g = h->reps[(size_t)r].g;
        const int zc = h->reps[(size_t)r].zc;
        for (int bz = 0; bz < (g.nz + zc - 1) / zc; ++bz)
            for (int by = 0; by < (g.ny + PS_TY - 1) / PS_TY; ++by)
                for (int bx = 0; bx < (g.nx + PS_TX - 1) / PS_TX; ++bx) v.push_back({r, bx, by, bz});
    }
    const size_t npsi = v.size() - nmu - nlb;
    // longest z chunks first: the block scheduler then ends the launch on short
    // blocks instead of starting a long one last
    auto planes = [&](const BatchBlock &b) {
        const Rep &r = h->reps[(size_t)b.rep];
        return std::min(r.zc, r.g.nz - b.bz * r.zc);
    };
    std::stable_sort(v.begin() + (std::ptrdiff_t)(nmu + nlb), v.end(),
                     [&](const BatchBlock &a, const BatchBlock &b) { return planes(a) > planes(b); });
    if ((int)nmu != h->b_nmu || (int)nlb != h->b_nlb || (int)npsi > h->b_npsi_cap) return FLB_EINVAL;
    h->b_npsi = (int)npsi;
    int rc = cuerr(cudaMemcpyAsync(h->b_mu, v.data(), nmu * sizeof(BatchBlock), cudaMemcpyHostToDevice, h->st));
    if (rc == FLB_OK)
        rc = cuerr(cudaMemcpyAsync(h->b_lb, v.data() + nmu, nlb * sizeof(BatchBlock), cudaMemcpyHostToDevice, h->st));
    if (rc == FLB_OK)
        rc = cuerr(cudaMemcpyAsync(h->b_psi, v.data() + nmu + nlb, npsi * sizeof(BatchBlock), cudaMemcpyHostToDevice,
                                   h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    h->b_lists_ok = rc == FLB_OK;
    return rc;
}

// Write the descriptor table for the current state and reset the device step counter.
int batch_upload_table(flb_handle *h)
{
    std::vector<BatchRep> &t = h->b_host;
    t.assign(h->reps.size(), BatchRep());
    for (size_t k = 0; k < h->reps.size(); ++k) {
        Rep &r = h->reps[k];
        BatchRep &d = t[k];
        const Geom &g = r.g;
        d.lb = lb_args(r, r.psi[r.pcur]);
        d.psi[0] = r.psi[r.pcur];
        d.psi[1] = r.psi[r.pcur ^ 1];
        d.psis = r.psis;
        d.E = r.E;
        d.A = (float)r.p.A;
        d.B = (float)r.p.B;
        d.K = (float)r.p.K;
        d.M = (float)r.p.M;
        d.heun = r.p.integrator == FLB_HEUN;
        d.advect = (r.p.coupling & FLB_COUPLE_ADVECT) ? 1 : 0;
        d.noise = r.p.kT > 0 && r.p.M > 0;
        d.mu_in = (r.p.coupling & FLB_COUPLE_FORCE) && r.p.force_grad != FLB_FORCE_STRESS;
        d.q15 = r.q == 15;
        d.zc = r.zc;
        d.pstep_tasks = k < h->p_pstep.size() ? h->p_pstep[k] : 0;
        const uint64_t pd[3] = {(uint64_t)g.px, (uint64_t)g.py, (uint64_t)g.pz};
        const uint64_t ps[2] = {(uint64_t)g.px * 4, (uint64_t)g.px * g.py * 4};
        const uint32_t pb[3] = {(uint32_t)(PS_TX + 8), (uint32_t)(PS_TY + 6), 1};
        for (int j = 0; j < 2; ++j)
            if (encode_tensor_map_f32(&d.map_psi[j], d.psi[j], 3, pd, ps, pb) != cudaSuccess) return FLB_ECUDA;
        if (d.heun && encode_tensor_map_f32(&d.map_psis, r.psis, 3, pd, ps, pb) != cudaSuccess) return FLB_ECUDA;
        const uint64_t ud[4] = {(uint64_t)g.px, (uint64_t)g.py, (uint64_t)g.pz, 3};
        const uint64_t us[3] = {(uint64_t)g.px * 4, (uint64_t)g.px * g.py * 4, (uint64_t)g.pn * 4};
        const uint32_t ub[4] = {(uint32_t)(PS_TX + 8), (uint32_t)(PS_TY + 2), 1, 3};
        if (encode_tensor_map_f32(&d.map_u, r.u, 4, ud, us, ub) != cudaSuccess) return FLB_ECUDA;
        const uint32_t mb[3] = {(uint32_t)(PS_TX + 8), (uint32_t)(PS_TY + 4), 1};
        if (encode_tensor_map_f32(&d.map_mu, r.mu, 3, pd, ps, mb) != cudaSuccess) return FLB_ECUDA;
    }
    int rc = cuerr(cudaMemcpyAsync(h->b_reps, t.data(), t.size() * sizeof(BatchRep), cudaMemcpyHostToDevice, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaMemsetAsync(h->b_dstep, 0, sizeof(long long), h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    return rc;
}

BatchLists batch_lists(flb_handle *h)
{
    BatchLists L;
    L.reps = h->b_reps;
    L.mu = h->b_mu;
    L.lb = h->b_lb;
    L.psi = h->b_psi;
    L.nmu = h->b_nmu;
    L.nlb = h->b_nlb;
    L.npsi = h->b_npsi;
    L.dstep = h->b_dstep;
    L.status = h->status;
    return L;
}

int batch_kernels_per_step(const flb_handle *h)
{
    const flb_params &p = h->reps[0].p;
    bool force = false;
    for (const Rep &r : h->reps) force |= (r.p.coupling & FLB_COUPLE_FORCE) != 0;
    // mu (when any replica is forced), collide-stream, velocity, psi stage(s), step counter
    return (force ? 1 : 0) + 1 + 1 + 1 + (p.integrator == FLB_HEUN ? 1 : 0) + 1;
}

// Every replica's step forms mu of psi^n for its force, so the batched FV
// stage 1 may read it instead of forming it.
bool batch_mu_in(const flb_handle *h)
{
    for (const Rep &r : h->reps)
        if (!(r.p.coupling & FLB_COUPLE_FORCE) || r.p.force_grad == FLB_FORCE_STRESS) return false;
    return true;
}

// Capture one batched step into a CUDA graph (once per handle).
int batch_capture(flb_handle *h)
{
    if (h->b_exec) return FLB_OK;
    bool ghost = false, force = false, noise = false;
    for (const Rep &r : h->reps) {
        ghost |= r.gamma_g != 0.f;
        force |= (r.p.coupling & FLB_COUPLE_FORCE) != 0;
        noise |= r.p.kT > 0 && r.p.M > 0;
    }
    const flb_params &p0 = h->reps[0].p;
    const BatchLists L = batch_lists(h);
    // the kernels' attributes are set by one launch outside the capture on a zero-block list
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return FLB_ECUDA;
    const cudaError_t e =
        launch_batch_step(L, p0.storage, ghost, force, 1, p0.integrator == FLB_HEUN, noise, batch_mu_in(h),
                          h->reps[0].q == 15, h->st);
    const cudaError_t e2 = cudaStreamEndCapture(h->st, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        return FLB_ECUDA;
    }
    if (cudaGraphInstantiate(&h->b_exec, gr, 0) != cudaSuccess) {
        cudaGraphDestroy(gr);
        h->b_exec = nullptr;
        return FLB_ECUDA;
    }
    h->b_graph = gr;
    return FLB_OK;
}

Rep *get_rep(flb_handle *h, int32_t rep)
{
    if (!h || rep < 0 || rep >= (int32_t)h->reps.size()) return nullptr;
    return &h->reps[(size_t)rep];
}

}  // namespace

namespace {
int step_batched(flb_handle *h, int64_t n)
{
    if (!batch_supported(h)) return FLB_EUNSUPPORTED;
    int rc = FLB_OK;
    if (!h->b_lists_ok) rc = batch_upload_lists(h);
    if (rc == FLB_OK) rc = batch_upload_table(h);
    if (rc == FLB_OK) rc = batch_capture(h);
    if (rc != FLB_OK) return rc;
    const int kps = batch_kernels_per_step(h);
    for (int64_t k = 0; k < n; ++k) {
        cudaEvent_t e0 = mark(h);
        if (cudaGraphLaunch(h->b_exec, h->st) != cudaSuccess) return FLB_ECUDA;
        h->launches += kps;
        span(h, 0, e0, mark(h), kps);
        for (Rep &r : h->reps) {
            r.cur ^= 1;
            r.pcur ^= 1;
            r.step += 1;
        }
        if (h->sample_every > 0 && h->sample_mask && h->reps[0].step % h->sample_every == 0)
            for (Rep &r : h->reps) {
                const int rs = sample_rep(h, r, h->sample_mask);
                if (rs != FLB_OK) return rs;
            }
    }
    return FLB_OK;
}

bool persist_supported(const flb_handle *h)
{
    if (!batch_supported(h)) return false;
    for (const Rep &r : h->reps)
        if (r.p.storage != FLB_F32_DEV) return false;
    return true;
}

// One step's task list: phase by phase, replica by replica, tile by tile; the
// need of a task counts the tasks of its replica listed before it.
int persist_build(flb_handle *h)
{
    std::vector<PTask> v;
    const size_t nr = h->reps.size();
    std::vector<int> need(nr, 0);
    for (int ph = 0; ph < PH_COUNT; ++ph)
        for (size_t k = 0; k < nr; ++k) {
            const Rep &r = h->reps[k];
            int c[PH_COUNT];
            persist_tiles(r.g, r.zc, r.p.coupling, r.p.integrator == FLB_HEUN ? 1 : 0, c);
            if (c[ph] == 0) continue;
            persist_tasks(v, (int)k, ph, r.g, r.zc, need[k]);
            need[k] += c[ph];
        }
    if (v.size() > h->p_cap) return FLB_EINVAL;
    h->p_pstep = need;
    h->p_ntask = (int)v.size();
    int rc = cuerr(cudaMemcpyAsync(h->p_tasks, v.data(), v.size() * sizeof(PTask), cudaMemcpyHostToDevice, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    h->p_ok = rc == FLB_OK;
    return rc;
}

// n steps of every replica, one cooperative launch per stretch between sampling steps.
int step_persistent(flb_handle *h, int64_t n)
{
    if (!persist_supported(h)) return FLB_EUNSUPPORTED;
    int rc = h->p_ok ? FLB_OK : persist_build(h);
    if (rc == FLB_OK) rc = batch_upload_table(h);  // descriptors of the current buffers; device step 0
    if (rc != FLB_OK) return rc;
    int64_t done = 0;
    while (done < n) {
        int64_t k = n - done;
        const int64_t st0 = h->reps[0].step;
        if (h->sample_every > 0 && h->sample_mask) k = std::min<int64_t>(k, h->sample_every - st0 % h->sample_every);
        k = std::min<int64_t>(k, 1 << 20);
        rc = cuerr(cudaMemsetAsync(h->p_ticket, 0, sizeof(unsigned), h->st));
        if (rc == FLB_OK) rc = cuerr(cudaMemsetAsync(h->p_abort, 0, sizeof(int), h->st));
        if (rc == FLB_OK) rc = cuerr(cudaMemsetAsync(h->p_done, 0, h->reps.size() * sizeof(unsigned), h->st));
        if (rc != FLB_OK) return rc;
        PersistArgs a;
        a.L = batch_lists(h);
        a.tasks = h->p_tasks;
        a.ntask = h->p_ntask;
        a.nsteps = (int)k;
        a.ds0 = done;
        a.ticket = h->p_ticket;
        a.done = h->p_done;
        a.abort = h->p_abort;
        a.status = h->status;
        a.wait_ns = h->wait_ns;
        cudaEvent_t e0 = mark(h);
        ++h->launches;
        if (launch_persist(a, h->reps[0].q == 15, h->st) != cudaSuccess) return FLB_ECUDA;
        span(h, 0, e0, mark(h), 1);
        for (Rep &r : h->reps) {
            r.cur ^= (int)(k & 1);
            r.pcur ^= (int)(k & 1);
            r.step += k;
        }
        done += k;
        if (h->sample_every > 0 && h->sample_mask && h->reps[0].step % h->sample_every == 0)
            for (Rep &r : h->reps) {
                const int rs = sample_rep(h, r, h->sample_mask);
                if (rs != FLB_OK) return rs;
            }
    }
    return FLB_OK;
}
}  // namespace

// window gather (flb_obs.cu)
namespace flb {
cudaError_t launch_window(const Geom &g, int q, int storage, const void *f, const float *psi, int x0, int y0, int z0,
                          int wx, int wy, int wz, float *out, cudaStream_t s);
}

extern "C" {

void flb_params_default(flb_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dim = 3;
    p->q = 19;
    p->nx = p->ny = p->nz = 32;
    p->rho0 = 1.0;
    p->tau = 0.8;
    p->gamma_bulk = NAN;
    p->gamma_ghost = 0.0;
    p->kT = 0.0;
    p->A = 0.05;
    p->B = 0.0;
    p->K = 0.04;
    p->M = 0.1;
    p->psi_scheme = FLB_FV;
    p->integrator = FLB_HEUN;
    p->storage = FLB_F32_DEV;
    p->coupling = FLB_COUPLE_FORCE | FLB_COUPLE_ADVECT;
    p->seed = 1;
    p->sq_kmax = 0;
    p->force_grad = FLB_FORCE_MATCHED;
    p->init = FLB_INIT_REST;
}

static bool valid_set(const flb_params *p, int32_t nrep)
{
    if (!p || nrep <= 0) return false;
    for (int32_t k = 0; k < nrep; ++k) {
        if (!valid(p[k])) return false;
        if (p[k].dim != p[0].dim || p[k].q != p[0].q || p[k].psi_scheme != p[0].psi_scheme ||
            p[k].integrator != p[0].integrator || p[k].storage != p[0].storage)
            return false;
    }
    return true;
}

size_t flb_workspace_bytes(const flb_params *p, int32_t nrep)
{
    if (!valid_set(p, nrep)) return 0;
    flb_handle h;
    h.reps.resize((size_t)nrep);
    for (int32_t k = 0; k < nrep; ++k) init_rep_consts(h.reps[(size_t)k], p[k]);
    return carve_all(h, nullptr);
}

int flb_init(const flb_params *p, int32_t nrep, void *dev_ws, size_t ws_bytes, void *cuda_stream, flb_handle **out)
{
    if (!out) return FLB_EINVAL;
    *out = nullptr;
    if (!valid_set(p, nrep) || !dev_ws || ((uintptr_t)dev_ws & 255)) return FLB_EINVAL;
    flb_handle *h = new (std::nothrow) flb_handle();
    if (!h) return FLB_EINVAL;
    h->reps.resize((size_t)nrep);
    for (int32_t k = 0; k < nrep; ++k) init_rep_consts(h->reps[(size_t)k], p[k]);
    const size_t need = carve_all(*h, nullptr);
    if (ws_bytes < need) {
        delete h;
        return FLB_ENOSPC;
    }
    h->ws = (char *)dev_ws;
    h->ws_bytes = ws_bytes;
    h->st = (cudaStream_t)cuda_stream;
    carve_all(*h, (char *)dev_ws);
    // zero the whole workspace: every replica at rest; then the equilibrium starts
    int rc = cuerr(cudaMemsetAsync(dev_ws, 0, need, h->st));
    for (Rep &r : h->reps) {
        if (rc != FLB_OK || r.p.init != FLB_INIT_EQUILIBRIUM) continue;
        const flb_params &p = r.p;
        float *psi = r.psi[r.pcur];
        rc = cuerr(launch_equilibrium_start(r.g, r.q, p.storage, lap_weights(r.dim, p.laplacian), p.rho0, p.kT, p.A,
                                            p.K, p.seed, r.f[r.cur], r.f[r.cur ^ 1], psi, h->st));
        if (rc != FLB_OK) break;
        // u: the velocity of the drawn populations (they sit where a step leaves them)
        LBArgs la = lb_args(r, psi);
        la.fout = r.f[r.cur];
        la.coupling = 0;
        rc = cuerr(r.dim == 2 ? launch_vel2(la, p.storage, h->st)
                              : r.q == 15 ? launch_vel15(la, p.storage, h->st) : launch_vel3(la, p.storage, h->st));
        if (rc == FLB_OK)
            rc = cuerr(cudaMemsetAsync(r.f[r.cur ^ 1], 0, (size_t)r.q * (size_t)r.g.n * (size_t)r.pop_elem, h->st));
    }
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return FLB_OK;
}

// dst[s] = (float)src[s], split over the host's cores for large fields
static void to_float(const double *src, float *dst, long long n)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const long long nt = n < (1 << 20) ? 1 : std::min<long long>(hw, 32);
    auto part = [&](long long t) {
        const long long a = n * t / nt, b = n * (t + 1) / nt;
        for (long long s = a; s < b; ++s) dst[s] = (float)src[s];
    };
    if (nt == 1) {
        part(0);
        return;
    }
    std::vector<std::thread> pool;
    for (long long t = 1; t < nt; ++t) pool.emplace_back(part, t);
    part(0);
    for (auto &th : pool) th.join();
}

int flb_set_fields(flb_handle *h, int32_t rep, const double *rho, const double *u, const double *psi)
{
    Rep *r = get_rep(h, rep);
    if (!r) return FLB_EINVAL;
    const Geom &g = r->g;
    const long long N = g.n;
    cudaStream_t st = h->st;
    // psi and u go up as interior FP32 fields, staged in the mu plane (free
    // scratch between steps), and are padded with their images on the device
    float *tmp = h->host_stage((size_t)N);
    auto put = [&](const double *src, float *dst) -> int {
        to_float(src, tmp, N);
        int rc = cuerr(cudaMemcpyAsync(r->mu, tmp, (size_t)N * 4, cudaMemcpyHostToDevice, st));
        if (rc == FLB_OK) rc = cuerr(launch_pad(g, r->mu, dst, st));
        ++h->launches;
        return rc == FLB_OK ? cuerr(cudaStreamSynchronize(st)) : rc;  // tmp is reused
    };
    int rc = psi ? put(psi, r->psi[r->pcur]) : cuerr(cudaMemsetAsync(r->psi[r->pcur], 0, (size_t)g.pn * 4, st));
    if (rc == FLB_OK && !u) rc = cuerr(cudaMemsetAsync(r->u, 0, (size_t)r->dim * g.pn * 4, st));
    for (int a = 0; a < r->dim && rc == FLB_OK && u; ++a) rc = put(u + (size_t)a * N, r->u + (size_t)a * g.pn);
    if (rc == FLB_OK && rho) {
        to_float(rho, tmp, N);
        rc = upload_padded(h, g, r->mu, tmp);  // padded rho in the mu plane for init_eq
    }
    if (rc != FLB_OK) return rc;
    const cudaError_t e = launch_init_eq(g, r->q, r->p.storage, rho ? r->mu : nullptr, r->u, (float)r->p.rho0,
                                         r->f[r->cur], st);
    ++h->launches;
    if (e != cudaSuccess) return FLB_ECUDA;
    return cuerr(cudaStreamSynchronize(st));
}

int flb_get_populations(flb_handle *h, int32_t rep, double *f)
{
    Rep *r = get_rep(h, rep);
    if (!r || !f) return FLB_EINVAL;
    std::vector<float> dev;
    const int rc = download_pops(h, *r, dev);
    if (rc != FLB_OK) return rc;
    const Geom &g = r->g;
    const long long N = g.n;
    for (int i = 0; i < r->q; ++i) {
        const int *c = cvec(r->q, i);
        const double wr = wgt(r->q, i) * r->p.rho0;
        for (int z = 0; z < g.nz; ++z)
            for (int y = 0; y < g.ny; ++y)
                for (int x = 0; x < g.nx; ++x) {
                    const long long src = g.sidx(wrapi(x - c[0], g.nx), wrapi(y - c[1], g.ny),
                                                 g.dim == 3 ? wrapi(z - c[2], g.nz) : 0);
                    f[(size_t)i * N + g.sidx(x, y, z)] = wr + (double)dev[(size_t)i * N + src];
                }
    }
    return FLB_OK;
}

int flb_set_populations(flb_handle *h, int32_t rep, const double *f)
{
    Rep *r = get_rep(h, rep);
    if (!r || !f) return FLB_EINVAL;
    std::vector<float> dev;
    phys_to_stored(*r, f, dev);
    const int rc = upload_pops(h, *r, dev);
    return rc == FLB_OK ? cuerr(cudaStreamSynchronize(h->st)) : rc;
}

// dst[s] = src[s] (FP32 to FP64), split over the host's cores for large fields
static void to_double(const float *src, double *dst, long long n)
{
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const long long nt = n < (1 << 20) ? 1 : std::min<long long>(hw, 32);
    auto part = [&](long long t) {
        const long long a = n * t / nt, b = n * (t + 1) / nt;
        for (long long s = a; s < b; ++s) dst[s] = (double)src[s];
    };
    if (nt == 1) {
        part(0);
        return;
    }
    std::vector<std::thread> pool;
    for (long long t = 1; t < nt; ++t) pool.emplace_back(part, t);
    part(0);
    for (auto &th : pool) th.join();
}

// psi and u: the interiors are gathered on the device into the spare population
// buffer (scratch between steps, >= 18 bytes per site), copied as N floats per
// field and converted on the host's cores
int flb_get_psi_u(flb_handle *h, int32_t rep, double *psi, double *u)
{
    Rep *r = get_rep(h, rep);
    if (!r) return FLB_EINVAL;
    const Geom &g = r->g;
    if (!psi && !u) return FLB_OK;
    float *scratch = (float *)r->f[r->cur ^ 1];
    const int nf = (psi ? 1 : 0) + (u ? r->dim : 0);
    int k = 0, rc = FLB_OK;
    if (psi) rc = cuerr(launch_unpad(g, r->psi[r->pcur], scratch + (size_t)g.n * k++, h->st));
    if (u)
        for (int a = 0; a < r->dim && rc == FLB_OK; ++a)
            rc = cuerr(launch_unpad(g, r->u + (size_t)a * g.pn, scratch + (size_t)g.n * k++, h->st));
    if (rc != FLB_OK) return rc;
    float *tmp = h->host_stage((size_t)g.n * nf);
    rc = cuerr(cudaMemcpyAsync(tmp, scratch, (size_t)g.n * nf * 4, cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    k = 0;
    if (psi) to_double(tmp + (size_t)g.n * k++, psi, g.n);
    if (u) to_double(tmp + (size_t)g.n * k, u, (long long)r->dim * g.n);
    return FLB_OK;
}

int flb_get_window(flb_handle *h, int32_t rep, int32_t x0, int32_t y0, int32_t z0, int32_t wx, int32_t wy,
                   int32_t wz, double *f, double *psi)
{
    Rep *r = get_rep(h, rep);
    if (!r || wx <= 0 || wy <= 0 || wz <= 0) return FLB_EINVAL;
    if (r->dim == 2 && wz != 1) return FLB_EINVAL;
    const long long W = (long long)wx * wy * wz;
    if (W > WIN_MAX) return FLB_ENOSPC;
    const Geom &g = r->g;
    const int xw = wrapi(((x0 % g.nx) + g.nx) % g.nx, g.nx), yw = ((y0 % g.ny) + g.ny) % g.ny,
              zw = ((z0 % g.nz) + g.nz) % g.nz;
    cudaError_t e = launch_window(g, r->q, r->p.storage, r->f[r->cur], r->psi[r->pcur], xw, yw, zw, wx, wy, wz,
                                  h->win, h->st);
    ++h->launches;
    if (e != cudaSuccess) return FLB_ECUDA;
    std::vector<float> buf((size_t)W * (r->q + 1));
    int rc = cuerr(cudaMemcpyAsync(buf.data(), h->win, buf.size() * 4, cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    if (f)
        for (int i = 0; i < r->q; ++i) {
            const double wr = wgt(r->q, i) * r->p.rho0;
            for (long long k = 0; k < W; ++k) f[i * W + k] = wr + (double)buf[(size_t)i * W + k];
        }
    if (psi)
        for (long long k = 0; k < W; ++k) psi[k] = buf[(size_t)r->q * W + k];
    return FLB_OK;
}

int flb_step(flb_handle *h, int64_t n)
{
    if (!h || n < 0) return FLB_EINVAL;
    const Range range("flb_step");
    if (h->mode == FLB_MODE_BATCHED) return n > 0 ? step_batched(h, n) : FLB_OK;
    if (h->mode == FLB_MODE_PERSISTENT) return n > 0 ? step_persistent(h, n) : FLB_OK;
    for (int64_t k = 0; k < n; ++k) {
        for (Rep &r : h->reps) {
            const int rc = step_rep(h, r);
            if (rc != FLB_OK) return rc;
            if (h->sample_every > 0 && h->sample_mask && r.step % h->sample_every == 0) {
                const int rs = sample_rep(h, r, h->sample_mask);
                if (rs != FLB_OK) return rs;
            }
        }
    }
    return FLB_OK;
}

namespace {
// Moment basis of the lattice (App. B leaves it open): Gram-Schmidt under
// <a, b> = sum_i w_i a_i b_i on the ordered monomials 1; c; c^2; 3c_x^2 - c^2;
// c_y^2 - c_z^2; c_x c_y; c_y c_z; c_z c_x; c^2 c; c_x(c_y^2 - c_z^2), c_y(c_z^2 - c_x^2),
// c_z(c_x^2 - c_y^2); c^4; c^2(3c_x^2 - c^2); c^2(c_y^2 - c_z^2) (D3Q19; D3Q15 ends
// c_x c_y c_z, c^4 after the c^2 c rows; D2Q9: 1; c; c^2; c_x^2 - c_y^2; c_x c_y;
// c^2 c; c^4), in plane order.
double mode_monomial(int dim, int q, int k, const int *cv)
{
    const double x = cv[0], y = cv[1], z = cv[2], c2 = x * x + y * y + z * z;
    if (dim == 2) {
        const double m[9] = {1, x, y, c2, x * x - y * y, x * y, c2 * x, c2 * y, c2 * c2};
        return m[k];
    }
    if (q == 15 && k >= 13) return k == 13 ? x * y * z : c2 * c2;
    const double m[19] = {1, x, y, z, c2, 3 * x * x - c2, y * y - z * z, x * y, y * z, z * x, c2 * x, c2 * y, c2 * z,
                          x * (y * y - z * z), y * (z * z - x * x), z * (x * x - y * y), c2 * c2,
                          c2 * (3 * x * x - c2), c2 * (y * y - z * z)};
    return m[k];
}

ModeBasis mode_basis(int dim, int q)
{
    double E[19][19];
    for (int k = 0; k < q; ++k) {
        for (int i = 0; i < q; ++i) E[k][i] = mode_monomial(dim, q, k, cvec(q, i));
        for (int l = 0; l < k; ++l) {
            double dot = 0.0, nl = 0.0;
            for (int i = 0; i < q; ++i) {
                dot += wgt(q, i) * E[k][i] * E[l][i];
                nl += wgt(q, i) * E[l][i] * E[l][i];
            }
            for (int i = 0; i < q; ++i) E[k][i] -= dot / nl * E[l][i];
        }
    }
    ModeBasis B;
    B.q = q;
    for (int k = 0; k < q; ++k)
        for (int i = 0; i < q; ++i) B.E[k * q + i] = (float)E[k][i];
    return B;
}
}  // namespace

int flb_mode_variances(flb_handle *h, int32_t rep, double *msq)
{
    Rep *r = get_rep(h, rep);
    if (!r || !msq) return FLB_EINVAL;
    const Geom &g = r->g;
    const int nb = (int)std::min<long long>(RED_MAX_BLOCKS, (g.n + 255) / 256);
    const cudaError_t e = launch_mode_msq(g, r->p.storage, mode_basis(r->dim, r->q), r->f[r->cur], h->red_partial,
                                          nb, h->red_out, h->st);
    h->launches += 2;
    if (e != cudaSuccess) return FLB_ECUDA;
    double out[NMSQ];
    int rc = cuerr(cudaMemcpyAsync(out, h->red_out, sizeof(out), cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    for (int k = 0; k < r->q; ++k) msq[k] = out[k] / (double)g.n;
    return out[NMSQ - 1] > 0.0 ? FLB_ENONFINITE : FLB_OK;
}

int flb_get_step(flb_handle *h, int32_t rep, int64_t *step)
{
    Rep *r = get_rep(h, rep);
    if (!r || !step) return FLB_EINVAL;
    *step = r->step;
    return FLB_OK;
}

int flb_moments(flb_handle *h, int32_t rep, double *totals, double *u2)
{
    Rep *r = get_rep(h, rep);
    if (!r) return FLB_EINVAL;
    const Geom &g = r->g;
    const int nb = (int)std::min<long long>(RED_MAX_BLOCKS, (g.n + 255) / 256);
    cudaError_t e = launch_totals(g, r->q, r->p.storage, r->f[r->cur], r->psi[r->pcur], r->u, h->red_partial, nb,
                                  h->red_out, h->st);
    h->launches += 2;
    if (e != cudaSuccess) return FLB_ECUDA;
    double out[NRED];
    int rc = cuerr(cudaMemcpyAsync(out, h->red_out, sizeof(out), cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    if (totals) {
        totals[0] = (double)g.n * r->p.rho0 + out[0];
        for (int a = 0; a < r->dim; ++a) totals[1 + a] = out[1 + a];
        totals[1 + r->dim] = out[4];
    }
    if (u2)
        for (int a = 0; a < r->dim; ++a) u2[a] = out[5 + a] / (double)g.n;
    const int st = take_status(h);
    if (st != FLB_OK) return st;
    return out[8] > 0 ? FLB_ENONFINITE : FLB_OK;
}

int flb_set_sampling(flb_handle *h, int32_t every_m, int32_t mask)
{
    if (!h || every_m < 0 || mask < 0 || mask > 7) return FLB_EINVAL;
    h->sample_every = every_m;
    h->sample_mask = mask;
    return FLB_OK;
}

int flb_sample(flb_handle *h, int32_t mask)
{
    if (!h || mask < 0 || mask > 7) return FLB_EINVAL;
    for (Rep &r : h->reps) {
        const int rc = sample_rep(h, r, mask);
        if (rc != FLB_OK) return rc;
    }
    return FLB_OK;
}

int64_t flb_structure_factor_size(flb_handle *h, int32_t rep, int32_t which)
{
    Rep *r = get_rep(h, rep);
    if (!r) return -1;
    if (which == FLB_SQ_PSI) return (int64_t)r->Kx * r->Ky * r->Kz;
    if (which == FLB_SQ_HEIGHT) return r->dim == 3 ? (int64_t)r->g.nx * r->g.ny : 0;
    if (which == FLB_SQ_DYNAMIC) return (int64_t)r->Kx * r->Ky * r->Kz * r->p.sq_lags;
    return -1;
}

int flb_structure_factor(flb_handle *h, int32_t rep, int32_t which, double *out, int64_t *nsamples)
{
    Rep *r = get_rep(h, rep);
    if (!r || !out || (which != FLB_SQ_PSI && which != FLB_SQ_HEIGHT && which != FLB_SQ_DYNAMIC)) return FLB_EINVAL;
    if (which == FLB_SQ_HEIGHT && r->dim != 3) return FLB_EINVAL;
    if (which == FLB_SQ_DYNAMIC && !r->dacc) return FLB_EINVAL;
    const int64_t cnt = flb_structure_factor_size(h, rep, which);
    const double *src = which == FLB_SQ_PSI ? r->sq : which == FLB_SQ_HEIGHT ? r->hsq : r->dacc;
    const int64_t ns = which == FLB_SQ_PSI ? r->sq_n : which == FLB_SQ_HEIGHT ? r->h_n : r->d_n;
    int rc = cuerr(cudaMemcpyAsync(out, src, (size_t)cnt * 8, cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    if (which == FLB_SQ_DYNAMIC) {
        const int64_t K = (int64_t)r->Kx * r->Ky * r->Kz;
        for (int64_t l = 0; l < r->p.sq_lags; ++l) {
            const int64_t nl = ns - l;  // samples with a partner l intervals earlier
            for (int64_t k = 0; k < K; ++k) out[l * K + k] = nl > 0 ? out[l * K + k] / (double)nl : 0.0;
        }
        if (nsamples) *nsamples = ns;
        return FLB_OK;
    }
    for (int64_t k = 0; k < cnt; ++k) out[k] = ns > 0 ? out[k] / (double)ns : 0.0;
    if (which == FLB_SQ_HEIGHT) out[0] = 0.0;  // the mean height carries no capillary mode
    if (nsamples) *nsamples = ns;
    return FLB_OK;
}

int flb_sq_reset(flb_handle *h, int32_t rep)
{
    if (!h) return FLB_EINVAL;
    for (int32_t k = 0; k < (int32_t)h->reps.size(); ++k) {
        if (rep >= 0 && k != rep) continue;
        Rep &r = h->reps[(size_t)k];
        int rc = cuerr(cudaMemsetAsync(r.sq, 0, (size_t)r.Kx * r.Ky * r.Kz * 8, h->st));
        if (rc == FLB_OK && r.hsq) rc = cuerr(cudaMemsetAsync(r.hsq, 0, (size_t)r.g.nx * r.g.ny * 8, h->st));
        if (rc == FLB_OK && r.dacc)
            rc = cuerr(cudaMemsetAsync(r.dacc, 0, (size_t)r.Kx * r.Ky * r.Kz * r.p.sq_lags * 8, h->st));
        if (rc != FLB_OK) return rc;
        r.sq_n = r.h_n = r.d_n = 0;
        r.dslot = -1;
    }
    return cuerr(cudaStreamSynchronize(h->st));
}

}  // extern "C"

namespace {
// Drop the batched mode's captured graph and block lists (rebuilt by the next batched step).
void batch_reset(flb_handle *h)
{
    if (h->b_exec) cudaGraphExecDestroy(h->b_exec);
    if (h->b_graph) cudaGraphDestroy(h->b_graph);
    h->b_exec = nullptr;
    h->b_graph = nullptr;
    h->b_lists_ok = false;
    h->p_ok = false;
}

std::string device_key()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
    for (char &c : name)
        if (c == ' ' || c == '\t' || c == '|') c = '_';
    return name + "|sm" + std::to_string(sms);
}

std::string rep_key(const Rep &r)
{
    char b[160];
    std::snprintf(b, sizeof b, "%dx%dx%d|q%d|s%d|i%d|n%d|a%d", r.g.nx, r.g.ny, r.g.nz, r.q, r.p.psi_scheme,
                  r.p.integrator, (r.p.kT > 0 && r.p.M > 0) ? 1 : 0, (r.p.coupling & FLB_COUPLE_ADVECT) ? 1 : 0);
    return b;
}

// Tuning cache: one "key<TAB>planes" line per tuned configuration; later lines win.
std::map<std::string, int> read_cache(const char *path)
{
    std::map<std::string, int> m;
    if (!path) return m;
    FILE *f = std::fopen(path, "r");
    if (!f) return m;
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char *tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        const int v = std::atoi(tab + 1);
        if (v >= PS_ZC_MIN && v <= 4096) m[line] = v;
    }
    std::fclose(f);
    return m;
}

void append_cache(const char *path, const std::string &key, int zc)
{
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s\t%d\n", key.c_str(), zc);
    std::fclose(f);
}

// Average device time of launch() over reps runs after one untimed run, in ms;
// < 0 if a launch failed.
float time_launches(flb_handle *h, const std::function<int()> &launch, int reps)
{
    if (launch() != FLB_OK) return -1.f;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1.f;
    float ms = -1.f;
    bool ok = cudaEventRecord(a, h->st) == cudaSuccess;
    for (int k = 0; ok && k < reps; ++k) ok = launch() == FLB_OK;
    ok = ok && cudaEventRecord(b, h->st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
         cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ok ? ms / reps : -1.f;
}

// Candidate planes per psi block for a box nz deep: every listed value below nz
// and the first one that covers the whole depth.
std::vector<int> zc_candidates(int nz)
{
    static const int kList[] = {4, 8, 16, 32, 64, 128, 256, 512};
    std::vector<int> v;
    for (int c : kList) {
        v.push_back(c);
        if (c >= nz) break;
    }
    return v;
}
}  // namespace

extern "C" {

int flb_get_tuning(flb_handle *h, int32_t rep, int32_t *psi_zchunk)
{
    Rep *r = get_rep(h, rep);
    if (!r || !psi_zchunk) return FLB_EINVAL;
    *psi_zchunk = r->zc;
    return FLB_OK;
}

int flb_set_tuning(flb_handle *h, int32_t rep, int32_t psi_zchunk)
{
    if (!h || psi_zchunk < PS_ZC_MIN || psi_zchunk > 4096) return FLB_EINVAL;
    if (rep == -1) {
        for (Rep &r : h->reps) r.zc = psi_zchunk;
    } else {
        Rep *r = get_rep(h, rep);
        if (!r) return FLB_EINVAL;
        r->zc = psi_zchunk;
    }
    batch_reset(h);
    return FLB_OK;
}

int flb_autotune(flb_handle *h, const char *cache_path, int32_t flags)
{
    if (!h || (flags & ~FLB_TUNE_FORCE)) return FLB_EINVAL;
    int rc = take_status(h);
    if (rc != FLB_OK) return rc;
    const bool force = (flags & FLB_TUNE_FORCE) != 0;
    const std::map<std::string, int> cache = force ? std::map<std::string, int>() : read_cache(cache_path);
    const std::string dk = device_key();
    const int reps = 3;
    if ((h->mode == FLB_MODE_BATCHED || h->mode == FLB_MODE_PERSISTENT) && batch_supported(h)) {
        // one value for every replica, timed on the batched psi launches
        std::string all;
        bool noise = false;
        int nzmax = 1;
        for (const Rep &r : h->reps) {
            all += rep_key(r) + ";";
            noise |= r.p.kT > 0 && r.p.M > 0;
            nzmax = std::max(nzmax, r.g.nz);
        }
        uint64_t hash = 1469598103934665603ull;  // FNV-1a over the replica keys
        for (unsigned char c : all) hash = (hash ^ c) * 1099511628211ull;
        char key[256];
        std::snprintf(key, sizeof key, "batched|%s|%zu|%016llx", dk.c_str(), h->reps.size(), (unsigned long long)hash);
        const bool heun = h->reps[0].p.integrator == FLB_HEUN;
        // the box depths present, deepest first
        std::vector<int> depths;
        for (const Rep &r : h->reps) depths.push_back(r.g.nz);
        std::sort(depths.begin(), depths.end(), std::greater<int>());
        depths.erase(std::unique(depths.begin(), depths.end()), depths.end());
        auto set_depth = [&](int nz, int zc) {
            for (Rep &r : h->reps)
                if (r.g.nz == nz) r.zc = zc;
        };
        auto time_all = [&](float &t) {
            batch_reset(h);
            int e = batch_upload_lists(h);
            if (e == FLB_OK) e = batch_upload_table(h);
            if (e != FLB_OK) return e;
            const BatchLists L = batch_lists(h);
            t = time_launches(h, [&]() {
                h->launches += heun ? 2 : 1;
                return cuerr(launch_batch_psi(L, heun, noise, batch_mu_in(h), h->reps[0].q == 15, h->st));
            }, reps);
            return t < 0.f ? (int)FLB_ECUDA : (int)FLB_OK;
        };
        const auto it = cache.find(key);
        if (it != cache.end()) {
            for (Rep &r : h->reps) r.zc = it->second;
            for (int nz : depths) {  // per-depth refinements, where tuned
                const auto d = cache.find(std::string(key) + "|nz" + std::to_string(nz));
                if (d != cache.end()) set_depth(nz, d->second);
            }
        } else {
            // one value for every replica first
            float tbest = 0.f;
            int best = PS_ZC;
            for (int zc : zc_candidates(nzmax)) {
                for (Rep &r : h->reps) r.zc = zc;
                float t = 0.f;
                if ((rc = time_all(t)) != FLB_OK) return rc;
                if (tbest == 0.f || t < tbest) {
                    tbest = t;
                    best = zc;
                }
            }
            for (Rep &r : h->reps) r.zc = best;
            append_cache(cache_path, key, best);
            // then each box depth on its own (the others held), over the chunk
            // sizes that split it evenly, ceil(nz / k); kept when 1% faster
            for (int nz : depths) {
                int dbest = best;
                for (int k = 1; k <= 16; ++k) {
                    const int zc = (nz + k - 1) / k;
                    if (zc < PS_ZC_MIN || zc == dbest || (k > 1 && zc == (nz + k - 2) / (k - 1))) continue;
                    set_depth(nz, zc);
                    float t = 0.f;
                    if ((rc = time_all(t)) != FLB_OK) return rc;
                    if (t < 0.99f * tbest) {
                        tbest = t;
                        dbest = zc;
                    }
                }
                set_depth(nz, dbest);
                append_cache(cache_path, std::string(key) + "|nz" + std::to_string(nz), dbest);
            }
        }
    } else {
        std::map<std::string, int> done;
        for (Rep &r : h->reps) {
            if (r.dim != 3 || general_path(r.p)) continue;
            const std::string key = "plain|" + dk + "|" + rep_key(r);
            auto d = done.find(key);
            if (d != done.end()) {
                r.zc = d->second;
                continue;
            }
            const auto it = cache.find(key);
            if (it != cache.end()) {
                r.zc = it->second;
            } else {
                float tbest = 0.f;
                int best = PS_ZC;
                for (int zc : zc_candidates(r.g.nz)) {
                    r.zc = zc;
                    const float t = time_launches(h, [&]() { return launch_psi_stages(h, r); }, reps);
                    if (t < 0.f) return FLB_ECUDA;
                    if (tbest == 0.f || t < tbest) {
                        tbest = t;
                        best = zc;
                    }
                }
                r.zc = best;
                append_cache(cache_path, key, best);
            }
            done[key] = r.zc;
        }
    }
    batch_reset(h);
    return take_status(h);
}

int flb_set_wait_limit(flb_handle *h, double seconds)
{
    if (!h || !(seconds >= 0.0) || seconds > 60.0) return FLB_EINVAL;
    h->wait_ns = (unsigned long long)(seconds * 1e9);
    return FLB_OK;
}

int flb_set_mode(flb_handle *h, int32_t mode)
{
    if (!h || (mode != FLB_MODE_PLAIN && mode != FLB_MODE_BATCHED && mode != FLB_MODE_PERSISTENT)) return FLB_EINVAL;
    h->mode = mode;
    for (Rep &r : h->reps) r.fused = 0;
    return FLB_OK;
}

int flb_set_psi_fused(flb_handle *h, int32_t on)
{
    if (!h) return FLB_EINVAL;
    if (on) {
        if (h->mode != FLB_MODE_PLAIN) return FLB_EUNSUPPORTED;
        for (const Rep &r : h->reps) {
            const flb_params &p = r.p;
            // FV: the D3Q19 operators; FD: either lattice (its operators are the SO stencils)
            const bool fv = p.psi_scheme == FLB_FV && r.q == 19, fd = p.psi_scheme == FLB_FD;
            if (r.dim != 3 || !(fv || fd) || p.integrator != FLB_HEUN || p.laplacian != FLB_LAP_SO)
                return FLB_EUNSUPPORTED;
        }
    }
    for (Rep &r : h->reps) r.fused = on ? 1 : 0;
    return FLB_OK;
}

size_t flb_state_bytes(flb_handle *h, int32_t rep)
{
    Rep *r = get_rep(h, rep);
    if (!r) return 0;
    const size_t N = (size_t)r->g.n;
    return 8 + (size_t)r->q * N * r->pop_elem + N * 4 + (size_t)r->dim * N * 4;
}

int flb_get_state(flb_handle *h, int32_t rep, void *host, size_t bytes)
{
    Rep *r = get_rep(h, rep);
    if (!r || !host) return FLB_EINVAL;
    if (bytes < flb_state_bytes(h, rep)) return FLB_ENOSPC;
    char *o = (char *)host;
    std::memcpy(o, &r->step, 8);
    o += 8;
    const size_t pb = (size_t)r->q * r->g.n * r->pop_elem;
    int rc = cuerr(cudaMemcpyAsync(o, r->f[r->cur], pb, cudaMemcpyDeviceToHost, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    o += pb;
    std::vector<float> tmp;
    rc = download_interior(h, r->g, r->psi[r->pcur], tmp);
    if (rc != FLB_OK) return rc;
    std::memcpy(o, tmp.data(), tmp.size() * 4);
    o += tmp.size() * 4;
    for (int a = 0; a < r->dim; ++a) {
        rc = download_interior(h, r->g, r->u + (size_t)a * r->g.pn, tmp);
        if (rc != FLB_OK) return rc;
        std::memcpy(o, tmp.data(), tmp.size() * 4);
        o += tmp.size() * 4;
    }
    return FLB_OK;
}

int flb_set_state(flb_handle *h, int32_t rep, const void *host, size_t bytes)
{
    Rep *r = get_rep(h, rep);
    if (!r || !host) return FLB_EINVAL;
    if (bytes < flb_state_bytes(h, rep)) return FLB_ENOSPC;
    const char *o = (const char *)host;
    std::memcpy(&r->step, o, 8);
    o += 8;
    const size_t pb = (size_t)r->q * r->g.n * r->pop_elem;
    int rc = cuerr(cudaMemcpyAsync(r->f[r->cur], o, pb, cudaMemcpyHostToDevice, h->st));
    if (rc == FLB_OK) rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    o += pb;
    const size_t N = (size_t)r->g.n;
    rc = upload_padded(h, r->g, r->psi[r->pcur], (const float *)o);
    o += N * 4;
    for (int a = 0; a < r->dim && rc == FLB_OK; ++a) {
        rc = upload_padded(h, r->g, r->u + (size_t)a * r->g.pn, (const float *)o);
        o += N * 4;
    }
    return rc;
}

int flb_synchronize(flb_handle *h)
{
    if (!h) return FLB_EINVAL;
    const int rc = cuerr(cudaStreamSynchronize(h->st));
    return rc != FLB_OK ? rc : take_status(h);
}

int64_t flb_launch_count(flb_handle *h) { return h ? h->launches : -1; }

int flb_set_profiling(flb_handle *h, int32_t on)
{
    if (!h) return FLB_EINVAL;
    const int rc = cuerr(cudaStreamSynchronize(h->st));
    h->profiling = on != 0;
    h->ev_used = 0;
    for (auto &s : h->spans) s.clear();
    for (auto &c : h->phase_launches) c = 0;
    return rc;
}

int flb_kernel_times(flb_handle *h, double *ms, int64_t *counts)
{
    if (!h || !ms) return FLB_EINVAL;
    const int rc = cuerr(cudaStreamSynchronize(h->st));
    if (rc != FLB_OK) return rc;
    for (int k = 0; k < 3; ++k) {
        double t = 0.0;
        for (auto &pr : h->spans[k]) {
            float x = 0.f;
            if (cudaEventElapsedTime(&x, pr.first, pr.second) != cudaSuccess) return FLB_ECUDA;
            t += x;
        }
        ms[k] = t;
        if (counts) counts[k] = h->phase_launches[k];
    }
    return FLB_OK;
}

namespace {
__global__ void gaussians_kernel(const PhiloxKey K, int64_t step, uint32_t stream, uint32_t site0, long long n,
                                 int nblocks, float *__restrict__ out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int b = 0; b < nblocks; ++b) {
        float G[8];
        normals<4>(K, step, site0 + (uint32_t)i, stream, (uint32_t)b, G);
        float *o = out + i * 8 * nblocks + 8 * b;
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = G[k];
    }
}
}  // namespace

int flb_gaussians(uint64_t seed, int64_t step, uint32_t stream, uint32_t site0, int64_t nsites, int32_t nblocks,
                  float *dev_out, void *cuda_stream)
{
    if (!dev_out || nsites < 0 || nblocks < 1 || nblocks > 16 || stream > 0xFFFFu ||
        (uint64_t)site0 + (uint64_t)nsites > (1ull << 32))
        return FLB_EINVAL;
    if (nsites == 0) return FLB_OK;
    const unsigned grid = (unsigned)((nsites + 255) / 256);
    gaussians_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(philox_key(seed), step, stream, site0, nsites,
                                                                   nblocks, dev_out);
    return cuerr(cudaGetLastError());
}

const char *flb_strerror(int code)
{
    switch (code) {
    case FLB_OK: return "ok";
    case FLB_EINVAL: return "invalid argument";
    case FLB_ENOSPC: return "workspace or buffer too small";
    case FLB_ECUDA: return "CUDA runtime error";
    case FLB_ENONFINITE: return "non-finite value in the fields";
    case FLB_ETIMEOUT: return "device-side wait timed out";
    case FLB_EUNSUPPORTED: return "unsupported in this build";
    default: return "unknown error";
    }
}

void flb_destroy(flb_handle *h) { delete h; }

}  // extern "C"
