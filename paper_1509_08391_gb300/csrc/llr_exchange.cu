// llr_exchange.cu -- replica exchange between overlapping energy intervals.
//
// Paper: Langfeld, Lucini, Pellegrini, Rago (arXiv:1509.08391), Sec. 2.5:
// for a pair of overlapping intervals (I1, I2) whose current configurations
// both have their energy in the common region, the configurations are
// exchanged with the Metropolis probability
//     min(1, exp((a_I1 - a_I2) (E_C1 - E_C2))).
//
// On the GPU a configuration is the link array a lattice state points to
// (LatState::off) together with its tracked energy, so an exchange swaps
// those two fields between the states of the pair: no link is copied.  The
// window, the slope, the Philox key and the sweep counter stay with the
// interval.  The pairs of one round are disjoint, so one thread decides and
// applies one pair with no synchronisation.
#include "llr_internal.h"

namespace llr {
namespace {

constexpr uint32_t kTagSwap = 13u;

__global__ void replica_exchange_kernel(LatState *lats, const int *pairs, int n_pairs,
                                        const double *a, uint32_t round, int *accepted)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_pairs) return;
    const int i1 = pairs[2 * k], i2 = pairs[2 * k + 1];
    LatState &s1 = lats[i1];
    LatState &s2 = lats[i2];
    const long long lo = s1.lo_fx > s2.lo_fx ? s1.lo_fx : s2.lo_fx;
    const long long hi = s1.hi_fx < s2.hi_fx ? s1.hi_fx : s2.hi_fx;
    const long long E1 = s1.E_fx, E2 = s2.E_fx;
    int take = 0;
    if (E1 >= lo && E1 <= hi && E2 >= lo && E2 <= hi) {
        // exponent in FP64; the energy difference is exact in fixed point
        const double x = (a[i1] - a[i2]) * ((double)(E1 - E2) * kInvFx);
        // 53-bit uniform in [0, 1) from the first two words of one Philox call
        const U4 w = philox4x32_10(0u, round, kTagSwap, 0u, s1.key0, s1.key1);
        const double u = ((double)(w.x >> 11) * 4294967296.0 + (double)w.y) *
                         (1.0 / 9007199254740992.0);
        take = (x >= 0.0 || u < exp(x)) ? 1 : 0;
    }
    if (take) {
        const unsigned long long off = s1.off;
        s1.off = s2.off;
        s2.off = off;
        s1.E_fx = E2;
        s2.E_fx = E1;
    }
    if (accepted) accepted[k] = take;
}

}  // namespace

cudaError_t launch_replica_exchange(LatState *lats, const int *pairs, int n_pairs,
                                    const double *a, uint32_t round, int *accepted,
                                    cudaStream_t s)
{
    if (n_pairs <= 0) return cudaSuccess;
    const int t = 128;
    replica_exchange_kernel<<<(n_pairs + t - 1) / t, t, 0, s>>>(lats, pairs, n_pairs, a, round,
                                                                 accepted);
    return cudaGetLastError();
}

}  // namespace llr
