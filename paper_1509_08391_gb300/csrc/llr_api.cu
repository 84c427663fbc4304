// llr_api.cu -- host side of the C ABI declared in include/llr.h: argument
// checking, device allocation of the lattice batch, stream-ordered launches
// and host <-> device marshalling.  All arithmetic of the method runs in the
// kernels of llr_chain.cu and llr_recon.cu.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/llr.h"
#include "llr_internal.h"

using llr::LatState;

struct llr_ctx {
    int n = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    float *d_theta = nullptr;
    size_t n_floats = 0;
    LatState *d_lat = nullptr;
    std::vector<LatState> h_lat;     // host copy of the static fields (geometry, window)
    double *d_a = nullptr, *d_mean = nullptr;
    int *d_int = nullptr;
    float *d_links = nullptr;        // staging for llr_get/set_links
    size_t links_cap = 0;
    int max_half = 0;
    int n_or = 4, block = 1;
    double beta_up = 1.5, beta_dn = 0.5;
    llr::LaunchCfg cfg;
    int last_launch[5] = {0, 0, 0, 0, 0};   // threads, fast math, ring, carve-out, grid
    unsigned long long wait_limit_ns = 20000000000ull;
    unsigned *d_sync = nullptr;      // work queue of the persistent kernel: 2 + n words
    int *d_order = nullptr;          // 0 .. n-1 (single-lattice launches point into it)
    int *d_step = nullptr;           // Robbins-Monro step counter of graph replays
    int *d_pairs = nullptr;          // replica-exchange pairs (n ints: at most n/2 pairs)
    // multicanonical weight: ln rho~ at the n + 1 edges, then the n slopes
    double *d_muca = nullptr;
    int muca_n = 0;
    double muca_e0 = 0.0, muca_de = 0.0, muca_a0 = 0.0;
    double *d_ehist = nullptr;       // energy history of llr_muca_sweep
    size_t ehist_cap = 0;
    // one captured Robbins-Monro step (memset, persistent kernel, step + 1)
    cudaGraphExec_t rm_graph = nullptr;
    int g_therm = -1, g_meas = -1, g_index0 = -1;
    int g_shape[4] = {0, 0, 0, 0};   // launch shape the graph was captured with
    double *g_a = nullptr, *g_hist = nullptr;
    cudaStream_t capture_stream = nullptr;
};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define LLR_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(LLR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool pow2_block(int b)
{
    return b >= 1 && b <= 32 && (b & (b - 1)) == 0;
}

llr::KernelArgs base_args(llr_handle h)
{
    llr::KernelArgs a;
    std::memset(&a, 0, sizeof(a));
    a.lats = h->d_lat;
    a.theta = h->d_theta;
    a.n_lat = h->n;
    a.n_or = h->n_or;
    a.block = h->block;
    a.beta_up = h->beta_up;
    a.beta_dn = h->beta_dn;
    a.class_mask = 0xFF;
    a.sync = h->d_sync;
    a.wait_limit_ns = h->wait_limit_ns;
    return a;
}

// Launch the persistent kernel with the handle's shape; remember the shape.
cudaError_t launch(llr_handle h, const llr::KernelArgs &a, cudaStream_t st)
{
    int grid = 0;
    const cudaError_t e = llr::launch_llr(a, h->cfg, st, &grid);
    if (e == cudaSuccess && grid > 0) {
        h->last_launch[0] = h->cfg.threads;
        h->last_launch[1] = h->cfg.fast_math ? 1 : 0;
        h->last_launch[2] = h->cfg.ring;
        h->last_launch[3] = h->cfg.carveout;
        h->last_launch[4] = grid;
    }
    return e;
}

// Error word of the persistent launches since the last check (nonzero: a
// bounded wait ran out in one of them); read and cleared.
int check_queue(llr_handle h)
{
    unsigned w = 0;
    LLR_CUDA(cudaMemcpyAsync(&w, h->d_sync, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    if (w) {
        LLR_CUDA(cudaMemsetAsync(h->d_sync, 0, sizeof(unsigned), h->stream));
        LLR_CUDA(cudaStreamSynchronize(h->stream));
        return fail(LLR_ERR_TIMEOUT, "a lattice's previous sweep was not done in time");
    }
    return LLR_OK;
}

int check_handle(llr_handle h)
{
    if (!h) return fail(LLR_ERR_ARG, "null handle");
    return LLR_OK;
}

int pull_states(llr_handle h, std::vector<LatState> &out)
{
    out.resize((size_t)h->n);
    LLR_CUDA(cudaMemcpyAsync(out.data(), h->d_lat, sizeof(LatState) * (size_t)h->n,
                             cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int ensure_links_buffer(llr_handle h, size_t n)
{
    if (h->links_cap >= n) return LLR_OK;
    if (h->d_links) cudaFree(h->d_links);
    h->d_links = nullptr;
    h->links_cap = 0;
    LLR_CUDA(cudaMalloc(&h->d_links, n * sizeof(float)));
    h->links_cap = n;
    return LLR_OK;
}

// The multicanonical weight table of eq. (2.10): tab[k] = ln rho~ at the
// edge e0 + k de (0 at k = 0) for k = 0..n, then the n slopes.
int muca_table(int n, double de, const double *a, std::vector<double> &tab)
{
    tab.assign(2 * (size_t)n + 1, 0.0);
    for (int k = 0; k < n; ++k) {
        if (!std::isfinite(a[k])) return fail(LLR_ERR_ARG, "non-finite slope");
        tab[(size_t)k + 1] = tab[(size_t)k] + a[k] * de;
        tab[(size_t)n + 1 + (size_t)k] = a[k];
    }
    return LLR_OK;
}

}  // namespace

int llr::set_last_error(int code, const char *msg)
{
    return fail(code, msg);
}

extern "C" {

const char *llr_last_error(void)
{
    return g_err.c_str();
}

int llr_init_lattice(llr_handle *out, const llr_config *cfg, void *cuda_stream)
{
    if (!out || !cfg) return fail(LLR_ERR_ARG, "null argument");
    *out = nullptr;
    const int n = cfg->n_lattices;
    if (n <= 0) return fail(LLR_ERR_ARG, "n_lattices must be positive");
    if (!cfg->L || !cfg->E_lo || !cfg->dE || !cfg->interval_id || !cfg->replica_id)
        return fail(LLR_ERR_ARG, "null configuration array");
    if (cfg->n_or < 0 || cfg->n_or > 64) return fail(LLR_ERR_ARG, "n_or must be in [0, 64]");
    if (!pow2_block(cfg->accept_block))
        return fail(LLR_ERR_ARG, "accept_block must be a power of two in [1, 32]");
    if (!std::isfinite(cfg->beta_up) || !std::isfinite(cfg->beta_dn))
        return fail(LLR_ERR_ARG, "beta_up / beta_dn must be finite");
    if (cfg->max_approach < 0) return fail(LLR_ERR_ARG, "max_approach must be >= 0");

    std::vector<LatState> st((size_t)n);
    size_t off = 0;
    int max_half = 0;
    for (int i = 0; i < n; ++i) {
        const int L = cfg->L[i];
        if (L < 2 || L > 64 || (L & 1))
            return fail(LLR_ERR_ARG, "lattice " + std::to_string(i) + ": L must be even, 2..64");
        const double lo = cfg->E_lo[i], w = cfg->dE[i];
        if (!std::isfinite(lo) || !std::isfinite(w) || !(w > 0.0))
            return fail(LLR_ERR_ARG, "lattice " + std::to_string(i) + ": bad window");
        const double hi = lo + w;
        if (std::fabs(lo) >= 2.0e9 || std::fabs(hi) >= 2.0e9)
            return fail(LLR_ERR_ARG, "lattice " + std::to_string(i) + ": window beyond +-2e9");
        LatState &s = st[(size_t)i];
        std::memset(&s, 0, sizeof(s));
        const long long V = (long long)L * L * L * L;
        s.L = L;
        s.half = (int)(V / 2);
        s.off = off;
        off += (size_t)(4 * V);
        off = (off + 31) & ~(size_t)31;   // 128-byte aligned lattices
        s.magic = (uint32_t)((4294967296ull + (unsigned long long)L - 1ull) / (unsigned long long)L);
        s.key0 = (uint32_t)cfg->seed ^ (uint32_t)cfg->interval_id[i];
        s.key1 = (uint32_t)(cfg->seed >> 32) ^ (uint32_t)cfg->replica_id[i];
        s.E_lo = lo;
        s.dE = w;
        s.lo_fx = (long long)std::ceil(lo * llr::kFx);
        s.hi_fx = (long long)std::floor(hi * llr::kFx);
        s.a = -1.0;
        if (s.half > max_half) max_half = s.half;
    }

    llr_ctx *h = new llr_ctx();
    h->n = n;
    h->stream = (cudaStream_t)cuda_stream;
    h->n_or = cfg->n_or;
    h->block = cfg->accept_block;
    h->beta_up = cfg->beta_up;
    h->beta_dn = cfg->beta_dn;
    h->h_lat = st;
    h->max_half = max_half;
    h->n_floats = off;
    cudaGetDevice(&h->device);
    *out = h;

    LLR_CUDA(cudaMalloc(&h->d_theta, off * sizeof(float)));
    LLR_CUDA(cudaMalloc(&h->d_lat, sizeof(LatState) * (size_t)n));
    LLR_CUDA(cudaMalloc(&h->d_a, sizeof(double) * (size_t)n));
    LLR_CUDA(cudaMalloc(&h->d_mean, sizeof(double) * (size_t)n));
    LLR_CUDA(cudaMalloc(&h->d_int, sizeof(int) * (size_t)(n + 1)));
    LLR_CUDA(cudaMalloc(&h->d_sync, sizeof(unsigned) * (size_t)(n + 2)));
    LLR_CUDA(cudaMemset(h->d_sync, 0, sizeof(unsigned) * (size_t)(n + 2)));
    LLR_CUDA(cudaMalloc(&h->d_order, sizeof(int) * (size_t)n));
    LLR_CUDA(cudaMalloc(&h->d_step, sizeof(int)));
    {
        std::vector<int> ord((size_t)n);
        for (int i = 0; i < n; ++i) ord[(size_t)i] = i;
        LLR_CUDA(cudaMemcpy(h->d_order, ord.data(), sizeof(int) * (size_t)n,
                            cudaMemcpyHostToDevice));
    }
    LLR_CUDA(cudaMemsetAsync(h->d_theta, 0, off * sizeof(float), h->stream));
    LLR_CUDA(cudaMemcpyAsync(h->d_lat, st.data(), sizeof(LatState) * (size_t)n,
                             cudaMemcpyHostToDevice, h->stream));
    LLR_CUDA(llr::launch_hot_start(h->d_lat, h->d_theta, n, max_half, h->stream));
    llr::KernelArgs a = base_args(h);
    a.program = llr::kProgResync;
    LLR_CUDA(launch(h, a, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    if (cfg->max_approach > 0) return llr_approach(h, cfg->max_approach, nullptr);
    return LLR_OK;
}

int llr_approach(llr_handle h, int max_sweeps, int *sweeps_out)
{
    if (int r = check_handle(h)) return r;
    if (max_sweeps < 0) return fail(LLR_ERR_ARG, "max_sweeps must be >= 0");
    llr::KernelArgs a = base_args(h);
    a.program = llr::kProgApproach;
    a.max_approach = max_sweeps;
    a.approach_sweeps = h->d_int;
    LLR_CUDA(launch(h, a, h->stream));
    if (sweeps_out)
        LLR_CUDA(cudaMemcpyAsync(sweeps_out, h->d_int, sizeof(int) * (size_t)h->n,
                                 cudaMemcpyDeviceToHost, h->stream));
    std::vector<LatState> st;
    if (int r = pull_states(h, st)) return r;
    if (int r = check_queue(h)) return r;
    for (int i = 0; i < h->n; ++i)
        if (st[(size_t)i].status == LLR_ERR_WINDOW)
            return fail(LLR_ERR_WINDOW, "lattice " + std::to_string(i) +
                                            " did not reach its window in " +
                                            std::to_string(max_sweeps) + " sweeps");
    return LLR_OK;
}

int llr_sweep(llr_handle h, const double *a_host, int n_sweeps, int measure, double *dE_sum_out)
{
    if (int r = check_handle(h)) return r;
    if (!a_host || n_sweeps < 0) return fail(LLR_ERR_ARG, "bad arguments");
    LLR_CUDA(cudaMemcpyAsync(h->d_a, a_host, sizeof(double) * (size_t)h->n,
                             cudaMemcpyHostToDevice, h->stream));
    llr::KernelArgs a = base_args(h);
    a.program = llr::kProgSweeps;
    a.n_therm = 0;
    a.n_meas = n_sweeps;
    a.measure = measure != 0;
    a.a_in = h->d_a;
    a.mean_out = h->d_mean;
    LLR_CUDA(launch(h, a, h->stream));
    if (dE_sum_out && measure)
        LLR_CUDA(cudaMemcpyAsync(dE_sum_out, h->d_mean, sizeof(double) * (size_t)h->n,
                                 cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return check_queue(h);
}

int llr_pass(llr_handle h, int kind, const double *a_host, int class_mask)
{
    if (int r = check_handle(h)) return r;
    if (kind < 0 || kind > 3)
        return fail(LLR_ERR_ARG, "kind must be 0 (heat-bath), 1 (overrelaxation), 2 "
                                 "(multicanonical) or 3 (end of a composite sweep)");
    if (class_mask < 1 || class_mask > 0xFF) return fail(LLR_ERR_ARG, "class_mask must be in 1..255");
    if (kind == 0 && !a_host) return fail(LLR_ERR_ARG, "heat-bath pass needs a");
    if (kind == 2 && !h->d_muca) return fail(LLR_ERR_ARG, "no multicanonical weight set");
    llr::KernelArgs a = base_args(h);
    a.program = llr::kProgPass;
    a.pass_kind = kind;
    a.class_mask = class_mask;
    if (kind == 2) {
        a.muca_lnr = h->d_muca;
        a.muca_a = h->d_muca + h->muca_n + 1;
        a.muca_n = h->muca_n;
        a.muca_e0 = h->muca_e0;
        a.muca_de = h->muca_de;
        a.muca_a0 = h->muca_a0;
    }
    if (a_host) {
        LLR_CUDA(cudaMemcpyAsync(h->d_a, a_host, sizeof(double) * (size_t)h->n,
                                 cudaMemcpyHostToDevice, h->stream));
        a.a_in = h->d_a;
    }
    LLR_CUDA(launch(h, a, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return check_queue(h);
}

int llr_rm_step_dev(llr_handle h, int n_therm, int n_meas, int rm_index, const double *a_in,
                    double *a_out, double *dE_mean_out)
{
    if (int r = check_handle(h)) return r;
    if (!a_in || !a_out || n_therm < 0 || n_meas < 1 || rm_index < 0)
        return fail(LLR_ERR_ARG, "bad arguments");
    llr::KernelArgs a = base_args(h);
    a.program = llr::kProgRM;
    a.n_therm = n_therm;
    a.n_meas = n_meas;
    a.measure = 1;
    a.rm_index = rm_index;
    a.a_in = a_in;
    a.a_out = a_out;
    a.mean_out = dE_mean_out;
    LLR_CUDA(launch(h, a, h->stream));
    return LLR_OK;
}

int llr_rm_step(llr_handle h, int n_therm, int n_meas, int rm_index, double *a_inout,
                double *dE_mean_out)
{
    if (int r = check_handle(h)) return r;
    if (!a_inout) return fail(LLR_ERR_ARG, "null a_inout");
    LLR_CUDA(cudaMemcpyAsync(h->d_a, a_inout, sizeof(double) * (size_t)h->n,
                             cudaMemcpyHostToDevice, h->stream));
    if (int r = llr_rm_step_dev(h, n_therm, n_meas, rm_index, h->d_a, h->d_a, h->d_mean))
        return r;
    LLR_CUDA(cudaMemcpyAsync(a_inout, h->d_a, sizeof(double) * (size_t)h->n,
                             cudaMemcpyDeviceToHost, h->stream));
    if (dE_mean_out)
        LLR_CUDA(cudaMemcpyAsync(dE_mean_out, h->d_mean, sizeof(double) * (size_t)h->n,
                                 cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    if (int r = check_queue(h)) return r;
    for (int i = 0; i < h->n; ++i)
        if (!std::isfinite(a_inout[i]))
            return fail(LLR_ERR_NUMERIC, "non-finite a for lattice " + std::to_string(i));
    return LLR_OK;
}

int llr_rm_run(llr_handle h, int n_therm, int n_meas, int rm_index0, int n_steps, double *a_dev,
               double *hist_dev)
{
    if (int r = check_handle(h)) return r;
    if (!a_dev || n_therm < 0 || n_meas < 1 || rm_index0 < 0 || n_steps < 0)
        return fail(LLR_ERR_ARG, "bad arguments");
    const int shape[4] = {h->cfg.threads, h->cfg.fast_math ? 1 : 0, h->cfg.ring, h->cfg.carveout};
    if (!h->rm_graph || h->g_therm != n_therm || h->g_meas != n_meas ||
        h->g_index0 != rm_index0 || h->g_a != a_dev || h->g_hist != hist_dev ||
        std::memcmp(shape, h->g_shape, sizeof(shape)) != 0) {
        if (h->rm_graph) cudaGraphExecDestroy(h->rm_graph);
        h->rm_graph = nullptr;
        if (!h->capture_stream)
            LLR_CUDA(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
        llr::KernelArgs a = base_args(h);
        a.program = llr::kProgRM;
        a.n_therm = n_therm;
        a.n_meas = n_meas;
        a.measure = 1;
        a.rm_index = rm_index0;
        a.a_in = a_dev;
        a.a_out = a_dev;
        a.step_dev = h->d_step;
        a.hist = hist_dev;
        llr::prime_launch(h->cfg);
        cudaGraph_t g;
        LLR_CUDA(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = launch(h, a, h->capture_stream);
        cudaError_t e2 = llr::launch_step_increment(h->d_step, h->capture_stream);
        cudaError_t e3 = cudaStreamEndCapture(h->capture_stream, &g);
        LLR_CUDA(e1);
        LLR_CUDA(e2);
        LLR_CUDA(e3);
        cudaError_t e4 = cudaGraphInstantiate(&h->rm_graph, g, 0);
        cudaGraphDestroy(g);
        LLR_CUDA(e4);
        h->g_therm = n_therm;
        h->g_meas = n_meas;
        h->g_index0 = rm_index0;
        h->g_a = a_dev;
        h->g_hist = hist_dev;
        std::memcpy(h->g_shape, shape, sizeof(shape));
    }
    LLR_CUDA(cudaMemsetAsync(h->d_step, 0, sizeof(int), h->stream));
    for (int k = 0; k < n_steps; ++k) LLR_CUDA(cudaGraphLaunch(h->rm_graph, h->stream));
    return LLR_OK;
}

int llr_rm_step_plain(llr_handle h, int n_therm, int n_meas, int rm_index, double *a_inout,
                      double *dE_mean_out)
{
    if (int r = check_handle(h)) return r;
    if (!a_inout || n_therm < 0 || n_meas < 1 || rm_index < 0)
        return fail(LLR_ERR_ARG, "bad arguments");
    LLR_CUDA(cudaMemcpyAsync(h->d_a, a_inout, sizeof(double) * (size_t)h->n,
                             cudaMemcpyHostToDevice, h->stream));
    // one lattice at a time, one launch of the same kernel per pass, resync, update
    llr::KernelArgs a = base_args(h);
    a.n_lat = 1;
    a.a_in = h->d_a;
    a.a_out = h->d_a;
    a.mean_out = h->d_mean;
    a.rm_index = rm_index;
    for (int i = 0; i < h->n; ++i) {
        a.order = h->d_order + i;
        a.program = llr::kProgBegin;
        LLR_CUDA(launch(h, a, h->stream));
        for (int j = 0; j < n_therm + n_meas; ++j) {
            a.program = llr::kProgPass;
            a.pass_kind = 0;
            LLR_CUDA(launch(h, a, h->stream));
            a.pass_kind = 1;
            for (int k = 0; k < h->n_or; ++k) LLR_CUDA(launch(h, a, h->stream));
            a.program = llr::kProgFinish;
            a.measure = j >= n_therm;
            LLR_CUDA(launch(h, a, h->stream));
        }
        a.program = llr::kProgUpdate;
        LLR_CUDA(launch(h, a, h->stream));
    }
    LLR_CUDA(cudaMemcpyAsync(a_inout, h->d_a, sizeof(double) * (size_t)h->n,
                             cudaMemcpyDeviceToHost, h->stream));
    if (dE_mean_out)
        LLR_CUDA(cudaMemcpyAsync(dE_mean_out, h->d_mean, sizeof(double) * (size_t)h->n,
                                 cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    if (int r = check_queue(h)) return r;
    for (int i = 0; i < h->n; ++i)
        if (!std::isfinite(a_inout[i]))
            return fail(LLR_ERR_NUMERIC, "non-finite a for lattice " + std::to_string(i));
    return LLR_OK;
}

int llr_replica_exchange(llr_handle h, int n_pairs, const int *pairs, const double *a_host,
                         uint32_t round, int *accepted_out)
{
    if (int r = check_handle(h)) return r;
    if (n_pairs < 0 || 2ll * n_pairs > (long long)h->n)
        return fail(LLR_ERR_ARG, "n_pairs must be in [0, n_lattices / 2]");
    if (n_pairs == 0) return LLR_OK;
    if (!pairs || !a_host) return fail(LLR_ERR_ARG, "null pairs or a");
    std::vector<char> used((size_t)h->n, 0);
    for (int k = 0; k < 2 * n_pairs; ++k) {
        const int i = pairs[k];
        if (i < 0 || i >= h->n) return fail(LLR_ERR_ARG, "pair index out of range");
        if (used[(size_t)i]) return fail(LLR_ERR_ARG, "lattice " + std::to_string(i) +
                                                          " appears in two pairs");
        used[(size_t)i] = 1;
    }
    for (int k = 0; k < n_pairs; ++k)
        if (h->h_lat[(size_t)pairs[2 * k]].L != h->h_lat[(size_t)pairs[2 * k + 1]].L)
            return fail(LLR_ERR_ARG, "the lattices of a pair must have the same L");
    for (int i = 0; i < h->n; ++i)
        if (!std::isfinite(a_host[i])) return fail(LLR_ERR_ARG, "non-finite a");
    if (!h->d_pairs) LLR_CUDA(cudaMalloc(&h->d_pairs, sizeof(int) * (size_t)h->n));
    LLR_CUDA(cudaMemcpyAsync(h->d_pairs, pairs, sizeof(int) * 2 * (size_t)n_pairs,
                             cudaMemcpyHostToDevice, h->stream));
    LLR_CUDA(cudaMemcpyAsync(h->d_a, a_host, sizeof(double) * (size_t)h->n,
                             cudaMemcpyHostToDevice, h->stream));
    LLR_CUDA(llr::launch_replica_exchange(h->d_lat, h->d_pairs, n_pairs, h->d_a, round, h->d_int,
                                          h->stream));
    if (accepted_out)
        LLR_CUDA(cudaMemcpyAsync(accepted_out, h->d_int, sizeof(int) * (size_t)n_pairs,
                                 cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_set_muca_weight(llr_handle h, int n, double e0, double de, const double *a_host,
                        double a0)
{
    if (int r = check_handle(h)) return r;
    if (n < 1 || !a_host || !std::isfinite(e0) || !std::isfinite(de) || !(de > 0.0) ||
        !std::isfinite(a0))
        return fail(LLR_ERR_ARG, "need n >= 1 finite slopes, finite e0, de > 0 and finite a0");
    std::vector<double> tab;
    if (int r = muca_table(n, de, a_host, tab)) return r;
    if (h->d_muca && h->muca_n != n) {
        LLR_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(h->d_muca);
        h->d_muca = nullptr;
    }
    if (!h->d_muca) LLR_CUDA(cudaMalloc(&h->d_muca, sizeof(double) * tab.size()));
    LLR_CUDA(cudaMemcpyAsync(h->d_muca, tab.data(), sizeof(double) * tab.size(),
                             cudaMemcpyHostToDevice, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    h->muca_n = n;
    h->muca_e0 = e0;
    h->muca_de = de;
    h->muca_a0 = a0;
    return LLR_OK;
}

int llr_muca_sweep(llr_handle h, int n_sweeps, double *E_out)
{
    if (int r = check_handle(h)) return r;
    if (n_sweeps < 0) return fail(LLR_ERR_ARG, "n_sweeps must be >= 0");
    if (!h->d_muca) return fail(LLR_ERR_ARG, "no multicanonical weight set");
    if (n_sweeps == 0) return LLR_OK;
    const size_t need = (size_t)n_sweeps * (size_t)h->n;
    if (E_out && h->ehist_cap < need) {
        LLR_CUDA(cudaStreamSynchronize(h->stream));
        cudaFree(h->d_ehist);
        h->d_ehist = nullptr;
        h->ehist_cap = 0;
        LLR_CUDA(cudaMalloc(&h->d_ehist, sizeof(double) * need));
        h->ehist_cap = need;
    }
    llr::KernelArgs a = base_args(h);
    a.program = llr::kProgMuca;
    a.n_therm = 0;
    a.n_meas = n_sweeps;
    a.muca_lnr = h->d_muca;
    a.muca_a = h->d_muca + h->muca_n + 1;
    a.muca_n = h->muca_n;
    a.muca_e0 = h->muca_e0;
    a.muca_de = h->muca_de;
    a.muca_a0 = h->muca_a0;
    a.e_hist = E_out ? h->d_ehist : nullptr;
    LLR_CUDA(launch(h, a, h->stream));
    if (E_out)
        LLR_CUDA(cudaMemcpyAsync(E_out, h->d_ehist, sizeof(double) * need, cudaMemcpyDeviceToHost,
                                 h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return check_queue(h);
}

int llr_energy(llr_handle h, double *E_out)
{
    if (int r = check_handle(h)) return r;
    if (!E_out) return fail(LLR_ERR_ARG, "null E_out");
    LLR_CUDA(llr::launch_energy_fp64(h->d_lat, h->d_theta, h->n, h->d_mean, h->stream));
    LLR_CUDA(cudaMemcpyAsync(E_out, h->d_mean, sizeof(double) * (size_t)h->n,
                             cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_tracked_energy(llr_handle h, double *E_out)
{
    if (int r = check_handle(h)) return r;
    if (!E_out) return fail(LLR_ERR_ARG, "null E_out");
    std::vector<LatState> st;
    if (int r = pull_states(h, st)) return r;
    for (int i = 0; i < h->n; ++i) E_out[i] = (double)st[(size_t)i].E_fx * llr::kInvFx;
    return LLR_OK;
}

int llr_get_links(llr_handle h, int lattice, float *out)
{
    if (int r = check_handle(h)) return r;
    if (!out || lattice < 0 || lattice >= h->n) return fail(LLR_ERR_ARG, "bad lattice or buffer");
    const int nl = 8 * h->h_lat[(size_t)lattice].half;
    if (int r = ensure_links_buffer(h, (size_t)nl)) return r;
    LLR_CUDA(llr::launch_to_canonical(h->d_lat + lattice, h->d_theta, h->d_links, nl, h->stream));
    LLR_CUDA(cudaMemcpyAsync(out, h->d_links, sizeof(float) * (size_t)nl, cudaMemcpyDeviceToHost,
                             h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_set_links(llr_handle h, int lattice, const float *in)
{
    if (int r = check_handle(h)) return r;
    if (!in || lattice < 0 || lattice >= h->n) return fail(LLR_ERR_ARG, "bad lattice or buffer");
    const int nl = 8 * h->h_lat[(size_t)lattice].half;
    if (int r = ensure_links_buffer(h, (size_t)nl)) return r;
    LLR_CUDA(cudaMemcpyAsync(h->d_links, in, sizeof(float) * (size_t)nl, cudaMemcpyHostToDevice,
                             h->stream));
    LLR_CUDA(llr::launch_from_canonical(h->d_lat + lattice, h->d_theta, h->d_links, nl, h->stream));
    // tracked energy from the FP64 plaquette sum of the new angles
    LLR_CUDA(llr::launch_energy_fp64(h->d_lat + lattice, h->d_theta, 1, h->d_mean, h->stream));
    LLR_CUDA(llr::launch_set_energy(h->d_lat + lattice, h->d_mean, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_get_sweep_counter(llr_handle h, int lattice, uint32_t *out)
{
    if (int r = check_handle(h)) return r;
    if (!out || lattice < 0 || lattice >= h->n) return fail(LLR_ERR_ARG, "bad lattice");
    LLR_CUDA(cudaMemcpyAsync(out, (char *)(h->d_lat + lattice) + offsetof(LatState, sweep),
                             sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_set_sweep_counter(llr_handle h, int lattice, uint32_t value)
{
    if (int r = check_handle(h)) return r;
    if (lattice < 0 || lattice >= h->n) return fail(LLR_ERR_ARG, "bad lattice");
    const uint32_t v = value;
    LLR_CUDA(cudaMemcpyAsync((char *)(h->d_lat + lattice) + offsetof(LatState, sweep), &v,
                             sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_stats(llr_handle h, double *out, int reset)
{
    if (int r = check_handle(h)) return r;
    if (!out) return fail(LLR_ERR_ARG, "null out");
    std::vector<LatState> st;
    if (int r = pull_states(h, st)) return r;
    for (int i = 0; i < h->n; ++i) {
        const LatState &s = st[(size_t)i];
        double *o = out + 8 * (size_t)i;
        o[0] = (double)s.hb_acc;
        o[1] = (double)s.hb_tot;
        o[2] = (double)s.or_acc;
        o[3] = (double)s.or_tot;
        o[4] = (double)s.caps;
        o[5] = s.max_drift;
        o[6] = (double)s.sweeps_done;
        o[7] = (double)s.status;
    }
    if (reset) {
        for (auto &s : st) {
            s.hb_acc = s.hb_tot = s.or_acc = s.or_tot = s.caps = 0ull;
            s.max_drift = 0.0;
            s.sweeps_done = 0ull;
        }
        LLR_CUDA(cudaMemcpyAsync(h->d_lat, st.data(), sizeof(LatState) * (size_t)h->n,
                                 cudaMemcpyHostToDevice, h->stream));
        LLR_CUDA(cudaStreamSynchronize(h->stream));
    }
    return LLR_OK;
}

int llr_status(llr_handle h, int *out)
{
    if (int r = check_handle(h)) return r;
    if (!out) return fail(LLR_ERR_ARG, "null out");
    std::vector<LatState> st;
    if (int r = pull_states(h, st)) return r;
    for (int i = 0; i < h->n; ++i) out[i] = st[(size_t)i].status;
    return check_queue(h);
}

int llr_set_kernel_config(llr_handle h, int threads, int fast_math)
{
    if (int r = check_handle(h)) return r;
    return llr_set_kernel_shape(h, threads, fast_math, h->cfg.ring, h->cfg.carveout);
}

int llr_set_kernel_shape(llr_handle h, int threads, int fast_math, int ring, int carveout)
{
    if (int r = check_handle(h)) return r;
    if (threads != 128 && threads != 160 && threads != 192 && threads != 256 && threads != 512)
        return fail(LLR_ERR_ARG, "threads must be 128, 160, 192, 256 or 512");
    if (ring != 1 && ring != 2 && ring != 4) return fail(LLR_ERR_ARG, "ring must be 1, 2 or 4");
    if (carveout != -1 && carveout != 50 && carveout != 75 && carveout != 100)
        return fail(LLR_ERR_ARG, "carveout must be -1 (default), 50, 75 or 100");
    h->cfg.threads = threads;
    h->cfg.fast_math = fast_math != 0;
    h->cfg.ring = ring;
    h->cfg.carveout = carveout;
    return LLR_OK;
}

int llr_get_last_launch(llr_handle h, int *out)
{
    if (int r = check_handle(h)) return r;
    if (!out) return fail(LLR_ERR_ARG, "null out");
    for (int k = 0; k < 5; ++k) out[k] = h->last_launch[k];
    return LLR_OK;
}

int llr_set_wait_limit(llr_handle h, unsigned long long ns)
{
    if (int r = check_handle(h)) return r;
    h->wait_limit_ns = ns;
    return LLR_OK;
}

size_t llr_state_bytes(llr_handle h)
{
    if (!h) return 0;
    return sizeof(LatState) * (size_t)h->n + sizeof(float) * h->n_floats;
}

int llr_save_state(llr_handle h, void *out)
{
    if (int r = check_handle(h)) return r;
    if (!out) return fail(LLR_ERR_ARG, "null buffer");
    char *p = (char *)out;
    LLR_CUDA(cudaMemcpyAsync(p, h->d_lat, sizeof(LatState) * (size_t)h->n, cudaMemcpyDeviceToHost,
                             h->stream));
    LLR_CUDA(cudaMemcpyAsync(p + sizeof(LatState) * (size_t)h->n, h->d_theta,
                             sizeof(float) * h->n_floats, cudaMemcpyDeviceToHost, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_load_state(llr_handle h, const void *in)
{
    if (int r = check_handle(h)) return r;
    if (!in) return fail(LLR_ERR_ARG, "null buffer");
    const LatState *st = (const LatState *)in;
    // replica exchange moves link arrays between lattices of the same L, so a
    // saved state may hold any arrangement of this handle's arrays among them
    std::vector<std::pair<unsigned long long, int>> own((size_t)h->n), saved((size_t)h->n);
    for (int i = 0; i < h->n; ++i) {
        const LatState &a = st[i], &b = h->h_lat[(size_t)i];
        if (a.L != b.L || a.half != b.half || a.key0 != b.key0 || a.key1 != b.key1 ||
            a.lo_fx != b.lo_fx || a.hi_fx != b.hi_fx)
            return fail(LLR_ERR_ARG, "state of lattice " + std::to_string(i) +
                                         " was saved from a different configuration");
        own[(size_t)i] = {b.off, b.L};
        saved[(size_t)i] = {a.off, a.L};
    }
    std::sort(own.begin(), own.end());
    std::sort(saved.begin(), saved.end());
    if (own != saved) return fail(LLR_ERR_ARG, "saved link arrays do not match this handle");
    LLR_CUDA(cudaMemcpyAsync(h->d_lat, in, sizeof(LatState) * (size_t)h->n, cudaMemcpyHostToDevice,
                             h->stream));
    LLR_CUDA(cudaMemcpyAsync(h->d_theta, (const char *)in + sizeof(LatState) * (size_t)h->n,
                             sizeof(float) * h->n_floats, cudaMemcpyHostToDevice, h->stream));
    LLR_CUDA(cudaStreamSynchronize(h->stream));
    return LLR_OK;
}

int llr_destroy(llr_handle h)
{
    if (!h) return LLR_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    cudaFree(h->d_theta);
    cudaFree(h->d_lat);
    cudaFree(h->d_a);
    cudaFree(h->d_mean);
    cudaFree(h->d_int);
    cudaFree(h->d_links);
    cudaFree(h->d_sync);
    cudaFree(h->d_order);
    cudaFree(h->d_step);
    cudaFree(h->d_pairs);
    cudaFree(h->d_muca);
    cudaFree(h->d_ehist);
    if (h->rm_graph) cudaGraphExecDestroy(h->rm_graph);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
    return LLR_OK;
}

// ---------------------------------------------------------------------------
// Reconstruction (stateless; default stream, synchronous)
// ---------------------------------------------------------------------------
namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};

int check_centres(int n, const double *c, const double *a)
{
    if (n < 1 || !c || !a) return fail(LLR_ERR_ARG, "need n >= 1 centres and slopes");
    for (int k = 0; k < n; ++k) {
        if (!std::isfinite(c[k]) || !std::isfinite(a[k]))
            return fail(LLR_ERR_ARG, "non-finite centre or slope");
        if (k > 0 && !(c[k] > c[k - 1])) return fail(LLR_ERR_ARG, "centres must ascend");
    }
    return LLR_OK;
}

// Samples of a multicanonical run on the device with ln rho~ at each, and the
// scratch of the reweighting kernels for up to kBetaBatch couplings a launch.
struct MucaSamples {
    static constexpr int kBetaBatch = 512;
    DevBuf buf;
    long long ns = 0;
    int gx = 1;
    double shift = 0.0;
    double *E = nullptr, *lr = nullptr, *beta = nullptr, *part = nullptr, *E1 = nullptr,
           *E2 = nullptr, *var = nullptr;
};

int muca_samples_init(MucaSamples &w, long long ns, const double *E, int n, double e0, double de,
                      const double *a)
{
    if (ns < 1 || !E) return fail(LLR_ERR_ARG, "need n_samples >= 1 samples");
    if (n < 1 || !a || !std::isfinite(e0) || !std::isfinite(de) || !(de > 0.0))
        return fail(LLR_ERR_ARG, "need n >= 1 finite slopes, finite e0 and de > 0");
    for (long long i = 0; i < ns; ++i)
        if (!std::isfinite(E[i])) return fail(LLR_ERR_ARG, "non-finite sample " + std::to_string(i));
    std::vector<double> tab;
    if (int r = muca_table(n, de, a, tab)) return r;
    int dev = 0, sms = 1;
    LLR_CUDA(cudaGetDevice(&dev));
    LLR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // sample blocks per coupling: two per SM, none without samples
    const long long tiles = (ns + 255) / 256;
    w.gx = (int)std::max(1LL, std::min(tiles, 2LL * sms));
    w.ns = ns;
    w.shift = e0;
    const int nb = MucaSamples::kBetaBatch;
    const size_t total = 2 * (size_t)ns + tab.size() + (size_t)nb * (4 * (size_t)w.gx + 4);
    LLR_CUDA(cudaMalloc(&w.buf.p, sizeof(double) * total));
    w.E = (double *)w.buf.p;
    w.lr = w.E + ns;
    double *dtab = w.lr + ns;
    w.beta = dtab + tab.size();
    w.part = w.beta + nb;
    w.E1 = w.part + 4 * (size_t)w.gx * nb;
    w.E2 = w.E1 + nb;
    w.var = w.E2 + nb;
    LLR_CUDA(cudaMemcpy(w.E, E, sizeof(double) * (size_t)ns, cudaMemcpyHostToDevice));
    LLR_CUDA(cudaMemcpy(dtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    LLR_CUDA(llr::launch_muca_lnrho(ns, w.E, dtab, dtab + n + 1, n, e0, de, w.lr,
                                    (int)std::min(tiles, 8LL * sms), nullptr));
    return LLR_OK;
}

// <E>, <E^2> and <E^2> - <E>^2 at nb couplings (host arrays; any output may
// be null), kBetaBatch couplings per launch.
int muca_moments(MucaSamples &w, int nb, const double *beta, double *E1, double *E2, double *var)
{
    for (int b0 = 0; b0 < nb; b0 += MucaSamples::kBetaBatch) {
        const int m = std::min(MucaSamples::kBetaBatch, nb - b0);
        LLR_CUDA(cudaMemcpy(w.beta, beta + b0, sizeof(double) * (size_t)m,
                            cudaMemcpyHostToDevice));
        LLR_CUDA(llr::launch_reweight(w.ns, w.E, w.lr, w.shift, m, w.beta, w.gx, w.part, w.E1,
                                      w.E2, w.var, nullptr));
        const size_t bytes = sizeof(double) * (size_t)m;
        if (E1) LLR_CUDA(cudaMemcpy(E1 + b0, w.E1, bytes, cudaMemcpyDeviceToHost));
        if (E2) LLR_CUDA(cudaMemcpy(E2 + b0, w.E2, bytes, cudaMemcpyDeviceToHost));
        if (var) LLR_CUDA(cudaMemcpy(var + b0, w.var, bytes, cudaMemcpyDeviceToHost));
    }
    return LLR_OK;
}

}  // namespace

int llr_muca_reweight(long long n_samples, const double *E, int n, double e0, double de,
                      const double *a, int n_beta, const double *beta, double *E_out,
                      double *E2_out)
{
    if (n_beta < 1 || !beta || !E_out || !E2_out) return fail(LLR_ERR_ARG, "bad beta arrays");
    for (int i = 0; i < n_beta; ++i)
        if (!std::isfinite(beta[i])) return fail(LLR_ERR_ARG, "non-finite beta");
    MucaSamples w;
    if (int r = muca_samples_init(w, n_samples, E, n, e0, de, a)) return r;
    return muca_moments(w, n_beta, beta, E_out, E2_out, nullptr);
}

int llr_muca_cv_peak(long long n_samples, const double *E, int n, double e0, double de,
                     const double *a, double beta_lo, double beta_hi, int n_grid, double tol,
                     double *out)
{
    if (!out || n_grid < 2 || !std::isfinite(beta_lo) || !std::isfinite(beta_hi) ||
        !(beta_hi > beta_lo) || !(tol > 0.0))
        return fail(LLR_ERR_ARG, "bad peak-search arguments");
    MucaSamples w;
    if (int r = muca_samples_init(w, n_samples, E, n, e0, de, a)) return r;
    // grid scan (Sec. 3.4), then golden-section search between the best
    // grid point's neighbours; every C_V evaluation is one reweighting
    std::vector<double> grid((size_t)n_grid), cv((size_t)n_grid);
    const double step = (beta_hi - beta_lo) / (double)(n_grid - 1);
    for (int i = 0; i < n_grid; ++i) grid[(size_t)i] = beta_lo + step * (double)i;
    if (int r = muca_moments(w, n_grid, grid.data(), nullptr, nullptr, cv.data())) return r;
    int best = 0;
    for (int i = 1; i < n_grid; ++i)
        if (cv[(size_t)i] > cv[(size_t)best]) best = i;
    double lo = grid[(size_t)std::max(best - 1, 0)];
    double hi = grid[(size_t)std::min(best + 1, n_grid - 1)];
    auto f = [&](double b, double &v) { return muca_moments(w, 1, &b, nullptr, nullptr, &v); };
    const double g = 0.6180339887498949;   // (sqrt 5 - 1) / 2
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo), f1 = 0.0, f2 = 0.0;
    if (int r = f(x1, f1)) return r;
    if (int r = f(x2, f2)) return r;
    for (int it = 0; it < 200 && hi - lo > tol; ++it) {
        if (f1 < f2) {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + g * (hi - lo);
            if (int r = f(x2, f2)) return r;
        } else {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - g * (hi - lo);
            if (int r = f(x1, f1)) return r;
        }
    }
    out[0] = 0.5 * (lo + hi);
    return f(out[0], out[1]);
}

int llr_muca_tunnellings(int n_steps, int n_chains, const double *E, double lo, double hi,
                         int *out)
{
    if (n_steps < 0 || n_chains < 1 || (n_steps > 0 && !E) || !out || std::isnan(lo) ||
        std::isnan(hi) || !(lo <= hi))
        return fail(LLR_ERR_ARG, "need n_steps >= 0, n_chains >= 1 and lo <= hi");
    const size_t ne = (size_t)n_steps * (size_t)n_chains;
    DevBuf b;
    LLR_CUDA(cudaMalloc(&b.p, sizeof(double) * ne + sizeof(int) * (size_t)n_chains));
    double *dE = (double *)b.p;
    int *dout = (int *)(dE + ne);
    if (ne) LLR_CUDA(cudaMemcpy(dE, E, sizeof(double) * ne, cudaMemcpyHostToDevice));
    LLR_CUDA(llr::launch_tunnellings(n_steps, n_chains, dE, lo, hi, dout, nullptr));
    LLR_CUDA(cudaMemcpy(out, dout, sizeof(int) * (size_t)n_chains, cudaMemcpyDeviceToHost));
    return LLR_OK;
}

int llr_reconstruct_lnrho(int n, const double *centres, const double *a, double *ln_rho_out)
{
    if (int r = check_centres(n, centres, a)) return r;
    if (!ln_rho_out) return fail(LLR_ERR_ARG, "null output");
    DevBuf b;
    LLR_CUDA(cudaMalloc(&b.p, sizeof(double) * 3 * (size_t)n));
    double *dc = (double *)b.p, *da = dc + n, *dl = da + n;
    LLR_CUDA(cudaMemcpy(dc, centres, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
    LLR_CUDA(cudaMemcpy(da, a, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
    LLR_CUDA(llr::launch_lnrho(n, dc, da, dl, nullptr));
    LLR_CUDA(cudaMemcpy(ln_rho_out, dl, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost));
    return LLR_OK;
}

int llr_observables(int n, const double *centres, const double *a, int n_beta,
                    const double *beta, double *lnZ_out, double *E_out, double *E2_out)
{
    if (int r = check_centres(n, centres, a)) return r;
    if (n_beta < 1 || !beta || !lnZ_out || !E_out || !E2_out)
        return fail(LLR_ERR_ARG, "bad beta arrays");
    DevBuf b;
    LLR_CUDA(cudaMalloc(&b.p, sizeof(double) * (3 * (size_t)n + 4 * (size_t)n_beta)));
    double *dc = (double *)b.p, *da = dc + n, *dl = da + n, *db = dl + n, *dz = db + n_beta,
           *d1 = dz + n_beta, *d2 = d1 + n_beta;
    LLR_CUDA(cudaMemcpy(dc, centres, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
    LLR_CUDA(cudaMemcpy(da, a, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
    LLR_CUDA(cudaMemcpy(db, beta, sizeof(double) * (size_t)n_beta, cudaMemcpyHostToDevice));
    LLR_CUDA(llr::launch_lnrho(n, dc, da, dl, nullptr));
    LLR_CUDA(llr::launch_observables(n, dc, dl, n_beta, db, dz, d1, d2, nullptr));
    LLR_CUDA(cudaMemcpy(lnZ_out, dz, sizeof(double) * (size_t)n_beta, cudaMemcpyDeviceToHost));
    LLR_CUDA(cudaMemcpy(E_out, d1, sizeof(double) * (size_t)n_beta, cudaMemcpyDeviceToHost));
    LLR_CUDA(cudaMemcpy(E2_out, d2, sizeof(double) * (size_t)n_beta, cudaMemcpyDeviceToHost));
    return LLR_OK;
}

int llr_cv_peak(int n, const double *centres, const double *a, double beta_lo, double beta_hi,
                int n_grid, double tol, double *out)
{
    if (int r = check_centres(n, centres, a)) return r;
    if (!out || n_grid < 2 || !(beta_hi > beta_lo) || !(tol > 0.0))
        return fail(LLR_ERR_ARG, "bad peak-search arguments");
    DevBuf b;
    LLR_CUDA(cudaMalloc(&b.p, sizeof(double) * (3 * (size_t)n + 2)));
    double *dc = (double *)b.p, *da = dc + n, *dl = da + n, *dout = dl + n;
    LLR_CUDA(cudaMemcpy(dc, centres, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
    LLR_CUDA(cudaMemcpy(da, a, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice));
    LLR_CUDA(llr::launch_lnrho(n, dc, da, dl, nullptr));
    LLR_CUDA(llr::launch_cv_peak(n, dc, dl, beta_lo, beta_hi, n_grid, tol, dout, nullptr));
    LLR_CUDA(cudaMemcpy(out, dout, sizeof(double) * 2, cudaMemcpyDeviceToHost));
    return LLR_OK;
}

}  // extern "C"
