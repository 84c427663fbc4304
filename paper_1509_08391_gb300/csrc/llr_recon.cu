// llr_recon.cu -- FP64 reconstruction of ln rho and of action observables
// from the Robbins-Monro slopes a_k.
//
// Paper: Langfeld, Lucini, Pellegrini, Rago (arXiv:1509.08391).
//   eqs. (2.6), (2.7)  ln rho(c_{k+1}) - ln rho(c_k) = (c_{k+1} - c_k) (a_k + a_{k+1}) / 2
//   eqs. (2.46), (2.47)    Z(beta) = sum_k w rho(c_k) e^{beta c_k},
//                    <E^m> = sum_k w c_k^m rho(c_k) e^{beta c_k} / Z
//   Sec. 3.4         C_V = <E^2> - <E>^2, beta_c at its maximum
//   Sec. 2.6, eq. (2.56)   multicanonical reweighting: a sample E_i of the run
//                    with weight 1/rho~ carries exp(beta E_i + ln rho~(E_i));
//                    tunnellings of a chain between the ends of the range
//
// Sizes are small (hundreds to thousands of intervals), so each quantity is
// one CTA: a block-wide FP64 scan for ln rho, log-sum-exp reductions for the
// observables, and a device-side grid scan + golden-section search for the
// C_V peak.
#include <string>

#include "../../include/llr.h"
#include "llr_internal.h"

// Scratch of llr_observables_noalloc: ln rho at up to LLR_NOALLOC_MAX_CENTRES
// interval centres, in a fixed device array that every GPU loading this
// library holds until the process exits.  Host code must not pass the symbol
// itself to a kernel (on the host it names a host-side stand-in); it uses the
// device address that cudaGetSymbolAddress returns.
static __device__ __align__(256) double g_noalloc_lnrho[LLR_NOALLOC_MAX_CENTRES];

namespace llr {
namespace {

constexpr int kT = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kT / 32; ++w) t += red[w];
    return t;
}

__device__ double block_max(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(kFull, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = red[0];
    for (int w = 1; w < kT / 32; ++w) t = fmax(t, red[w]);
    return t;
}

// Inclusive block scan of the trapezium increments, chunk by chunk.
__device__ void lnrho_scan(int n, const double *c, const double *a, double *out)
{
    __shared__ double buf[kT];
    __shared__ double carry;
    if (threadIdx.x == 0) carry = 0.0;
    __syncthreads();
    for (int base = 0; base < n; base += kT) {
        const int k = base + threadIdx.x;
        // increment arriving at centre k (0 for k = 0)
        double inc = 0.0;
        if (k > 0 && k < n) inc = 0.5 * (c[k] - c[k - 1]) * (a[k - 1] + a[k]);
        buf[threadIdx.x] = inc;
        __syncthreads();
        for (int o = 1; o < kT; o <<= 1) {
            const double y = threadIdx.x >= o ? buf[threadIdx.x - o] : 0.0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (k < n) out[k] = carry + buf[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) carry += buf[kT - 1];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kT) lnrho_kernel(int n, const double *c, const double *a,
                                                   double *out)
{
    lnrho_scan(n, c, a, out);
}

// (ln Z, <E>, <E^2>) at coupling beta; ln rho given.  Every thread returns them.
__device__ void moments_at(int n, const double *c, const double *lr, double beta, double *red,
                           double &lnZ, double &E1, double &E2)
{
    double m = -INFINITY;
    for (int k = threadIdx.x; k < n; k += kT) m = fmax(m, lr[k] + beta * c[k]);
    m = block_max(m, red);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = threadIdx.x; k < n; k += kT) {
        const double e = exp(lr[k] + beta * c[k] - m);
        s0 += e;
        s1 += c[k] * e;
        s2 += c[k] * c[k] * e;
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    const double w = n > 1 ? (c[n - 1] - c[0]) / (double)(n - 1) : 1.0;
    lnZ = m + log(w * s0);
    E1 = s1 / s0;
    E2 = s2 / s0;
}

__global__ void __launch_bounds__(kT) observables_kernel(int n, const double *c,
                                                         const double *lr, const double *beta,
                                                         double *lnZ, double *E1, double *E2)
{
    __shared__ double red[kT / 32];
    double z, e1, e2;
    moments_at(n, c, lr, beta[blockIdx.x], red, z, e1, e2);
    if (threadIdx.x == 0) {
        lnZ[blockIdx.x] = z;
        E1[blockIdx.x] = e1;
        E2[blockIdx.x] = e2;
    }
}

__device__ double cv_at(int n, const double *c, const double *lr, double beta, double *red)
{
    double z, e1, e2;
    moments_at(n, c, lr, beta, red, z, e1, e2);
    return e2 - e1 * e1;
}

__global__ void __launch_bounds__(kT) cv_peak_kernel(int n, const double *c, const double *lr,
                                                     double blo, double bhi, int n_grid,
                                                     double tol, double *out)
{
    __shared__ double red[kT / 32];
    int best = 0;
    double best_cv = -INFINITY;
    for (int i = 0; i < n_grid; ++i) {
        const double b = n_grid > 1 ? blo + (bhi - blo) * (double)i / (double)(n_grid - 1) : blo;
        const double v = cv_at(n, c, lr, b, red);
        if (v > best_cv) {
            best_cv = v;
            best = i;
        }
    }
    const double step = n_grid > 1 ? (bhi - blo) / (double)(n_grid - 1) : 0.0;
    double lo = blo + step * (double)(best > 0 ? best - 1 : 0);
    double hi = blo + step * (double)(best < n_grid - 1 ? best + 1 : n_grid - 1);
    const double g = 0.6180339887498949;   // (sqrt 5 - 1) / 2
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = cv_at(n, c, lr, x1, red), f2 = cv_at(n, c, lr, x2, red);
    for (int it = 0; it < 200 && hi - lo > tol; ++it) {
        if (f1 < f2) {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + g * (hi - lo);
            f2 = cv_at(n, c, lr, x2, red);
        } else {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - g * (hi - lo);
            f1 = cv_at(n, c, lr, x1, red);
        }
    }
    const double b = 0.5 * (lo + hi);
    const double v = cv_at(n, c, lr, b, red);
    if (threadIdx.x == 0) {
        out[0] = b;
        out[1] = v;
    }
}

// ---------------------------------------------------------------------------
// Multicanonical reweighting (Sec. 2.6, eq. (2.56)).  The moments at beta are
// log-space sums over all samples; they run over d = E - shift (shift = the
// table start, close to the samples), so that <E^2> - <E>^2 keeps its digits.

// ln rho~ of eq. (2.10) at E: lnr[k] = ln rho~(e0 + k de), slope a[k] on
// [e0 + k de, e0 + (k + 1) de), the first / last slope beyond the table.
__device__ __forceinline__ double lnrho_piecewise(const double *lnr, const double *a, int n,
                                                  double e0, double de, double E)
{
    const double q = fmin(fmax(floor((E - e0) / de), 0.0), (double)(n - 1));
    const int k = (int)q;
    return lnr[k] + a[k] * (E - (e0 + (double)k * de));
}

__global__ void __launch_bounds__(kT) muca_lnrho_kernel(long long ns, const double *E,
                                                        const double *lnr, const double *a,
                                                        int n, double e0, double de,
                                                        double *out)
{
    const long long stride = (long long)gridDim.x * kT;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < ns; i += stride)
        out[i] = lnrho_piecewise(lnr, a, n, e0, de, E[i]);
}

// Block (x, y): coupling beta[y] over the samples of kT-wide tiles x,
// x + gridDim.x, ...  Each thread keeps a running maximum m of the exponent
// and rescales its sums when it grows; the block then brings its threads to
// the block maximum M.  Writes (M, s0, s1, s2), s_j = sum d^j exp(x - M).
__global__ void __launch_bounds__(kT) reweight_partial_kernel(long long ns, const double *E,
                                                              const double *lr, double shift,
                                                              const double *beta, double *part)
{
    __shared__ double red[kT / 32];
    const double b = beta[blockIdx.y];
    double m = -INFINITY, s0 = 0.0, s1 = 0.0, s2 = 0.0;
    const long long stride = (long long)gridDim.x * kT;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < ns; i += stride) {
        const double e_i = E[i];
        const double x = b * e_i + lr[i];
        if (x > m) {
            const double r = exp(m - x);      // 0 on a thread's first sample
            s0 *= r;
            s1 *= r;
            s2 *= r;
            m = x;
        }
        const double w = exp(x - m);
        const double d = e_i - shift;
        s0 += w;
        s1 += d * w;
        s2 += d * d * w;
    }
    const double M = block_max(m, red);
    const double r = m == -INFINITY ? 0.0 : exp(m - M);
    s0 = block_sum(s0 * r, red);
    s1 = block_sum(s1 * r, red);
    s2 = block_sum(s2 * r, red);
    if (threadIdx.x == 0) {
        double *p = part + 4 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x);
        p[0] = M;
        p[1] = s0;
        p[2] = s1;
        p[3] = s2;
    }
}

// One block per coupling: combine the gx partials of reweight_partial_kernel.
// E1 = <E>, var = <E^2> - <E>^2, E2 = <E^2> (any of them may be null).
__global__ void __launch_bounds__(kT) reweight_combine_kernel(int gx, const double *part,
                                                              double shift, double *E1,
                                                              double *E2, double *var)
{
    __shared__ double red[kT / 32];
    const double *p = part + 4 * (size_t)blockIdx.x * gx;
    double m = -INFINITY;
    for (int j = threadIdx.x; j < gx; j += kT) m = fmax(m, p[4 * j]);
    m = block_max(m, red);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int j = threadIdx.x; j < gx; j += kT) {
        const double mj = p[4 * j];
        if (mj == -INFINITY) continue;        // a block without samples
        const double r = exp(mj - m);
        s0 += r * p[4 * j + 1];
        s1 += r * p[4 * j + 2];
        s2 += r * p[4 * j + 3];
    }
    s0 = block_sum(s0, red);
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    if (threadIdx.x == 0) {
        const double u = s1 / s0, v = s2 / s0 - u * u, e1 = shift + u;
        if (E1) E1[blockIdx.x] = e1;
        if (var) var[blockIdx.x] = v;
        if (E2) E2[blockIdx.x] = e1 * e1 + v;
    }
}

// Tunnellings of each chain (Sec. 2.6): E[t][c] in time order t; a passage
// from E < lo to E > hi or back counts once.  One thread per chain, the
// loads of a time step coalesced across chains.
__global__ void __launch_bounds__(kT) tunnelling_kernel(int n_steps, int n_chains,
                                                        const double *E, double lo, double hi,
                                                        int *out)
{
    const int c = blockIdx.x * kT + threadIdx.x;
    if (c >= n_chains) return;
    int count = 0, last = 0;
    for (int t = 0; t < n_steps; ++t) {
        const double e = E[(size_t)t * n_chains + c];
        if (e < lo) {
            count += last == 1;
            last = -1;
        } else if (e > hi) {
            count += last == -1;
            last = 1;
        }
    }
    out[c] = count;
}

}  // namespace

cudaError_t launch_muca_lnrho(long long ns, const double *E, const double *lnr, const double *a,
                              int n, double e0, double de, double *out, int grid,
                              cudaStream_t s)
{
    muca_lnrho_kernel<<<grid, kT, 0, s>>>(ns, E, lnr, a, n, e0, de, out);
    return cudaGetLastError();
}

cudaError_t launch_reweight(long long ns, const double *E, const double *lr, double shift,
                            int n_beta, const double *beta, int gx, double *part, double *E1,
                            double *E2, double *var, cudaStream_t s)
{
    if (n_beta <= 0) return cudaSuccess;
    reweight_partial_kernel<<<dim3(gx, n_beta), kT, 0, s>>>(ns, E, lr, shift, beta, part);
    reweight_combine_kernel<<<n_beta, kT, 0, s>>>(gx, part, shift, E1, E2, var);
    return cudaGetLastError();
}

cudaError_t launch_tunnellings(int n_steps, int n_chains, const double *E, double lo, double hi,
                               int *out, cudaStream_t s)
{
    tunnelling_kernel<<<(n_chains + kT - 1) / kT, kT, 0, s>>>(n_steps, n_chains, E, lo, hi, out);
    return cudaGetLastError();
}

cudaError_t launch_lnrho(int n, const double *c, const double *a, double *out, cudaStream_t s)
{
    lnrho_kernel<<<1, kT, 0, s>>>(n, c, a, out);
    return cudaGetLastError();
}

cudaError_t launch_observables(int n, const double *c, const double *lr, int n_beta,
                               const double *beta, double *lnZ, double *E1, double *E2,
                               cudaStream_t s)
{
    if (n_beta <= 0) return cudaSuccess;
    observables_kernel<<<n_beta, kT, 0, s>>>(n, c, lr, beta, lnZ, E1, E2);
    return cudaGetLastError();
}

cudaError_t launch_cv_peak(int n, const double *c, const double *lr, double beta_lo,
                           double beta_hi, int n_grid, double tol, double *out, cudaStream_t s)
{
    cv_peak_kernel<<<1, kT, 0, s>>>(n, c, lr, beta_lo, beta_hi, n_grid, tol, out);
    return cudaGetLastError();
}

}  // namespace llr

namespace {

// Device address of the scratch array in the current device's context,
// looked up on every call (a cheap table lookup once the module is loaded):
// a cached address would dangle after the context is destroyed and created
// again (cudaDeviceReset, or the primary context released and retained).
int noalloc_scratch(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_lnrho);
    if (e != cudaSuccess || !p)
        return llr::set_last_error(LLR_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") +
                                                  cudaGetErrorString(e)).c_str());
    *out = (double *)p;
    return LLR_OK;
}

}  // namespace

extern "C" int llr_observables_noalloc(int n, const double *centres, const double *a,
                                       int n_beta, const double *beta, double *lnZ_out,
                                       double *E_out, double *E2_out, void *cuda_stream)
{
    if (n < 1 || n > LLR_NOALLOC_MAX_CENTRES)
        return llr::set_last_error(LLR_ERR_ARG, ("n must be in 1.." +
                                                 std::to_string(LLR_NOALLOC_MAX_CENTRES) +
                                                 " for llr_observables_noalloc").c_str());
    if (n_beta < 1 || !centres || !a || !beta || !lnZ_out || !E_out || !E2_out)
        return llr::set_last_error(LLR_ERR_ARG, "null device buffer or n_beta < 1");
    double *scratch = nullptr;
    if (int r = noalloc_scratch(&scratch)) return r;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // every call writes ln rho at all n centres before the observables read
    // them, so the scratch needs no clearing between calls
    cudaError_t e = llr::launch_lnrho(n, centres, a, scratch, s);
    if (e == cudaSuccess)
        e = llr::launch_observables(n, centres, scratch, n_beta, beta, lnZ_out, E_out, E2_out, s);
    if (e != cudaSuccess)
        return llr::set_last_error(LLR_ERR_CUDA, (std::string("launch: ") +
                                                  cudaGetErrorString(e)).c_str());
    return LLR_OK;
}
