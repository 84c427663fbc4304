// llr_chain.cu -- the window-restricted Monte Carlo of 4-D compact U(1) on
// sm_103a: checkerboard staple sums, heat-bath and overrelaxation proposals,
// the sequential window-accept scan, the fresh energy and the Robbins-Monro
// update, for a batch of independent (interval, replica) lattices.
//
// Paper: Langfeld, Lucini, Pellegrini, Rago (arXiv:1509.08391).
//   Sec. 3.1      action E = sum_P cos(theta_P), plaquette angle
//                 theta_munu(x) = theta_mu(x) + theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x)
//   eqs. kk7-kk10 weight exp(-a E) on the closed window [E_lo, E_lo + dE],
//                 dE_meas = E - E_lo - dE/2
//   Algorithm 1   n_therm + n_meas sweeps, measure after n_therm
//   eq. kk21      a <- a + 12 <<dE>> / (dE^2 (n + 1))
//
// Design (one CTA owns one lattice for the whole launch):
//   * links are float32 angles, SoA by (direction, site parity), sites of a
//     parity in lexicographic order: theta[off + (2 mu + p) * V/2 + s/2];
//   * a class (mu, p) is updated in chunks of NT consecutive links: every
//     thread builds the 6 staples of its link from 18 neighbour angles and
//     draws its proposal (von Mises heat-bath, Best & Fisher 1979, or the
//     reflection theta' = -theta - 2 alpha), giving dE in FP32;
//   * dE goes to int64 fixed point (2^-32); each warp forms inclusive
//     prefix sums; warp 0 then walks the chunk in link order, deciding each
//     block of B links with the restricted Metropolis rule
//     dist(E + dE_block) <= dist(E), using a ballot to find the first
//     rejected block among 32 speculatively accepted ones;
//   * accepted angles are written back; after 1 + n_or passes the CTA sums
//     the 6V plaquettes (exact float32 angle sums + cosf, fixed-point
//     accumulation) and resynchronises the tracked energy.
#include <cstdio>

#include "llr_internal.h"

namespace llr {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Best & Fisher (1979) von Mises sampler, density ~ exp(kappa cos X).
// tau = 1 + sqrt(1 + 4 k^2), rho = (tau - sqrt(2 tau)) / (2 k) (rewritten
// without cancellation), r = (1 + rho^2) / (2 rho).  Per attempt:
// z = cos(pi u1), f = (1 + r z) / (r + z), c = k (r - f); accept if
// c (2 - c) > u2 or ln(c / u2) + 1 - c >= 0; X = +-acos(f) by u3.  acos(f) is
// evaluated as 2 asin(sqrt((1-f)/2)) or pi - 2 asin(sqrt((1+f)/2)) with
// 1 -+ f formed without cancellation, so small and near-pi angles keep
// full float precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool von_mises(float kappa, uint32_t c0, uint32_t c1, uint32_t c2,
                                          uint32_t k0, uint32_t k1, float &X)
{
    if (fabsf(kappa) < 1e-6f) {
        const U4 w = philox4x32_10(c0, c1, c2, 0u, k0, k1);
        X = kPi * (2.0f * u01(w.x) - 1.0f);
        return true;
    }
    const float k = fabsf(kappa);
    const float sq = sqrtf(fmaf(4.0f * k, k, 1.0f));
    const float tau = 1.0f + sq;
    const float rho = 2.0f * k * tau / ((sq + 1.0f) * (tau + sqrtf(2.0f * tau)));
    const float r = (1.0f + rho * rho) / (2.0f * rho);
    const float omr = 1.0f - rho;
    const float rm1 = omr * omr / (2.0f * rho);   // r - 1
    for (int att = 0; att < kSamplerMaxAttempts; ++att) {
        const U4 w = philox4x32_10(c0, c1, c2, (uint32_t)att, k0, k1);
        const float u1 = u01(w.x), u2 = u01(w.y), u3 = u01(w.z);
        const float z = cospif(u1);
        const float den = r + z;
        const float f = (1.0f + r * z) / den;
        const float c = k * (rm1 + (1.0f - f));
        if (c * (2.0f - c) - u2 > 0.0f || logf(c / u2) + 1.0f - c >= 0.0f) {
            float mag;
            if (f >= 0.0f) {
                const float sh = sinpif(0.5f * u1);
                const float g = rm1 * 2.0f * sh * sh / den;            // 1 - f
                mag = 2.0f * asinf(fminf(sqrtf(0.5f * g), 1.0f));
            } else {
                const float ch = cospif(0.5f * u1);
                const float hp = (r + 1.0f) * 2.0f * ch * ch / den;    // 1 + f
                mag = kPi - 2.0f * asinf(fminf(sqrtf(0.5f * hp), 1.0f));
            }
            float x = u3 > 0.5f ? mag : -mag;
            if (kappa < 0.0f) x = wrap_angle(x + kPi);
            X = x;
            return true;
        }
    }
    return false;
}

template <bool FAST>
__device__ __forceinline__ void sin_cos(float x, float *s, float *c)
{
    if (FAST)
        __sincosf(x, s, c);
    else
        sincosf(x, s, c);
}

// Coordinates of the h-th site of parity p (lexicographic, x0 fastest).
__device__ __forceinline__ int decode_half(int h, int p, int L, uint32_t magic, int x[4])
{
    const int n = 2 * h;
    int q = (int)__umulhi((uint32_t)n, magic);
    const int x0e = n - q * L;
    int q2 = (int)__umulhi((uint32_t)q, magic);
    x[1] = q - q2 * L;
    const int q3 = (int)__umulhi((uint32_t)q2, magic);
    x[2] = q2 - q3 * L;
    x[3] = q3;
    const int b = (p + x[1] + x[2] + x[3]) & 1;
    x[0] = x0e + b;
    return n + b;
}

// Staple sum S = sum_j exp(i phi_j) of link theta_MU(x), x of parity p:
// forward  phi = theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x)
// backward phi = theta_nu(x-nu) - theta_nu(x-nu+mu) - theta_mu(x-nu)
// so that the link's local energy is sum_j cos(theta + phi_j) = Re(e^{i theta} S).
template <int MU, bool FAST>
__device__ __forceinline__ void staple_sum(const float *__restrict__ th, int half, int L,
                                           const int x[4], int s, int p, float &Sr, float &Si)
{
    const int st[4] = {1, L, L * L, L * L * L};
    const int dmu = (x[MU] == L - 1) ? -(L - 1) * st[MU] : st[MU];
    const int spmu = s + dmu;
    const int q = p ^ 1;
    const float *thmu_q = th + (2 * MU + q) * half;
    Sr = 0.0f;
    Si = 0.0f;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == MU) continue;
        const int dnf = (x[nu] == L - 1) ? -(L - 1) * st[nu] : st[nu];
        const int dnb = (x[nu] == 0) ? (L - 1) * st[nu] : -st[nu];
        const int spnu = s + dnf;
        const int smnu = s + dnb;
        const int smnu_pmu = smnu + dmu;
        const float *thnu_p = th + (2 * nu + p) * half;
        const float *thnu_q = th + (2 * nu + q) * half;
        const float a1 = __ldg(thnu_q + (spmu >> 1));      // theta_nu(x+mu)
        const float a2 = __ldg(thmu_q + (spnu >> 1));      // theta_mu(x+nu)
        const float a3 = __ldg(thnu_p + (s >> 1));         // theta_nu(x)
        const float b1 = __ldg(thnu_p + (smnu_pmu >> 1));  // theta_nu(x-nu+mu)
        const float b2 = __ldg(thmu_q + (smnu >> 1));      // theta_mu(x-nu)
        const float b3 = __ldg(thnu_q + (smnu >> 1));      // theta_nu(x-nu)
        const float pf = a1 - a2 - a3;
        const float pb = b3 - b1 - b2;
        float sf, cf, sb, cb;
        sin_cos<FAST>(pf, &sf, &cf);
        sin_cos<FAST>(pb, &sb, &cb);
        Sr += cf + cb;
        Si += sf + sb;
    }
}

template <int NT>
struct Smem {
    LatState st;
    long long P[NT];
    long long bs[NT];
    unsigned endmask[NT / 32];
    unsigned accmask[NT / 32];
    long long red[NT / 32];
    unsigned long long acc_cnt;
    unsigned long long cap_cnt;
};

// One checkerboard class (MU, p).  kind 0: heat-bath at slope a_f with
// Philox tag `tag`; kind 1: overrelaxation.
template <int MU, int NT, bool FAST>
__device__ void class_update(Smem<NT> &sm, float *__restrict__ th, int p, int kind, float a_f,
                             uint32_t tag, int B)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic, V = 2u * (uint32_t)half;
    const uint32_t k0 = sm.st.key0, k1 = sm.st.key1, sweep = sm.st.sweep;
    float *own = th + (2 * MU + p) * half;
    const int nchunk = (half + NT - 1) / NT;
    for (int ch = 0; ch < nchunk; ++ch) {
        const int h = ch * NT + tid;
        const bool valid = h < half;
        float thn = 0.0f;
        long long d = 0;
        if (valid) {
            int x[4];
            const int s = decode_half(h, p, L, magic, x);
            float Sr, Si;
            staple_sum<MU, FAST>(th, half, L, x, s, p, Sr, Si);
            const float t0 = own[h];
            float so, co;
            sin_cos<FAST>(t0, &so, &co);
            const float e_old = co * Sr - so * Si;
            const float alpha = atan2f(Si, Sr);
            if (kind == 0) {
                const float Sabs = sqrtf(Sr * Sr + Si * Si);
                float X;
                const uint32_t link = (uint32_t)MU * V + (uint32_t)s;
                if (von_mises(-a_f * Sabs, link, sweep, tag, k0, k1, X)) {
                    thn = wrap_angle(X - alpha);
                } else {
                    thn = t0;
                    atomicAdd(&sm.cap_cnt, 1ull);
                }
            } else {
                thn = wrap_angle(-t0 - 2.0f * alpha);
            }
            float sn, cn;
            sin_cos<FAST>(thn, &sn, &cn);
            const float e_new = cn * Sr - sn * Si;
            d = to_fx(e_new - e_old);
        }
        // warp-inclusive prefix sums of the fixed-point dE
        long long P = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, P, o);
            if (lane >= o) P += y;
        }
        const int bstart = lane & ~(B - 1);
        const long long Pprev = __shfl_sync(kFull, P, bstart > 0 ? bstart - 1 : 0);
        const long long bsum = P - (bstart > 0 ? Pprev : 0ll);
        const bool isend = valid && (((lane & (B - 1)) == B - 1) || h == half - 1);
        const unsigned em = __ballot_sync(kFull, isend);
        sm.P[tid] = P;
        sm.bs[tid] = bsum;
        if (lane == 0) sm.endmask[warp] = em;
        __syncthreads();
        if (warp == 0) {
            // sequential Metropolis accept of the chunk's blocks in link order
            long long E = sm.st.E_fx;
            const long long lo = sm.st.lo_fx, hi = sm.st.hi_fx;
            for (int g = 0; g < NT / 32; ++g) {
                unsigned rem = sm.endmask[g];
                unsigned acc = 0u;
                const long long Pk = sm.P[g * 32 + lane];
                const long long bk = sm.bs[g * 32 + lane];
                long long base = 0;
                while (rem) {
                    const long long Ea = E + (Pk - base);
                    const long long Eb = Ea - bk;
                    const bool mine = (rem >> lane) & 1u;
                    const bool viol = mine && (dist_fx(Ea, lo, hi) > dist_fx(Eb, lo, hi));
                    const unsigned vm = __ballot_sync(kFull, viol);
                    if (vm == 0u) {
                        const int last = 31 - __clz(rem);
                        E += __shfl_sync(kFull, Pk, last) - base;
                        acc |= rem;
                        rem = 0u;
                    } else {
                        const int j = __ffs(vm) - 1;
                        acc |= rem & ((1u << j) - 1u);
                        const long long Pj = __shfl_sync(kFull, Pk, j);
                        const long long bj = __shfl_sync(kFull, bk, j);
                        E += (Pj - bj) - base;   // energy before the rejected block
                        base = Pj;               // skip its contribution
                        rem &= ~((2u << j) - 1u);
                    }
                }
                if (lane == 0) sm.accmask[g] = acc;
            }
            if (lane == 0) sm.st.E_fx = E;
        }
        __syncthreads();
        // write back the accepted proposals
        bool accepted = false;
        if (valid) {
            const unsigned e = sm.endmask[warp] & ~((1u << lane) - 1u);
            const int eb = __ffs(e) - 1;
            accepted = (sm.accmask[warp] >> eb) & 1u;
            if (accepted) own[h] = thn;
        }
        const unsigned am = __ballot_sync(kFull, accepted);
        if (lane == 0 && am) atomicAdd(&sm.acc_cnt, (unsigned long long)__popc(am));
    }
    __syncthreads();
}

template <int NT, bool FAST>
__device__ void full_pass(Smem<NT> &sm, float *th, int kind, float a_f, uint32_t tag, int B,
                          int class_mask = 0xFF)
{
    if (threadIdx.x == 0) sm.acc_cnt = 0ull;
    __syncthreads();
#pragma unroll 1
    for (int cls = 0; cls < 8; ++cls) {
        if (!((class_mask >> cls) & 1)) continue;
        const int p = cls & 1;
        switch (cls >> 1) {
            case 0: class_update<0, NT, FAST>(sm, th, p, kind, a_f, tag, B); break;
            case 1: class_update<1, NT, FAST>(sm, th, p, kind, a_f, tag, B); break;
            case 2: class_update<2, NT, FAST>(sm, th, p, kind, a_f, tag, B); break;
            default: class_update<3, NT, FAST>(sm, th, p, kind, a_f, tag, B); break;
        }
    }
    if (threadIdx.x == 0) {
        const unsigned long long n =
            (unsigned long long)__popc(class_mask & 0xFF) * (unsigned long long)sm.st.half;
        if (kind == 0) {
            sm.st.hb_acc += sm.acc_cnt;
            sm.st.hb_tot += n;
        } else {
            sm.st.or_acc += sm.acc_cnt;
            sm.st.or_tot += n;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// cos of the plaquette angle a + b - c - d of four float angles: the angle is
// formed exactly as hi + lo, cos(hi + lo) = cos(hi) - sin(hi) lo.
__device__ __forceinline__ float plaquette_cos(float a, float b, float c, float d)
{
    float s1, e1, s2, e2, hi, e3;
    two_sum(a, b, s1, e1);
    two_sum(c, d, s2, e2);
    two_sum(s1, -s2, hi, e3);
    const float lo = (e1 - e2) + e3;
    float sn, cs;
    sincosf(hi, &sn, &cs);
    return cs - sn * lo;
}

// Fresh energy of the CTA's lattice in fixed point: sum over the 6 V
// plaquettes, exact int64 accumulation and reduction.
template <int NT>
__device__ long long fresh_energy_fx(Smem<NT> &sm, const float *__restrict__ th)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic;
    const int V = 2 * half;
    const int st[4] = {1, L, L * L, L * L * L};
    long long acc = 0;
    for (int s = tid; s < V; s += NT) {
        int x[4];
        int q = (int)__umulhi((uint32_t)s, magic);
        x[0] = s - q * L;
        int q2 = (int)__umulhi((uint32_t)q, magic);
        x[1] = q - q2 * L;
        const int q3 = (int)__umulhi((uint32_t)q2, magic);
        x[2] = q2 - q3 * L;
        x[3] = q3;
        const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
        const int hs = s >> 1;
        float t[4];
        int sp[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            t[mu] = __ldg(th + (2 * mu + p) * half + hs);
            sp[mu] = s + ((x[mu] == L - 1) ? -(L - 1) * st[mu] : st[mu]);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                const float tnu_xmu = __ldg(th + (2 * nu + (p ^ 1)) * half + (sp[mu] >> 1));
                const float tmu_xnu = __ldg(th + (2 * mu + (p ^ 1)) * half + (sp[nu] >> 1));
                acc += to_fx(plaquette_cos(t[mu], tnu_xmu, tmu_xnu, t[nu]));
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if (lane == 0) sm.red[warp] = acc;
    __syncthreads();
    long long tot = 0;
    if (tid == 0)
        for (int w = 0; w < NT / 32; ++w) tot += sm.red[w];
    return tot;   // valid in thread 0 only
}

// Resync after a composite sweep; thread 0 updates the state.
template <int NT>
__device__ void end_of_sweep(Smem<NT> &sm, const float *th, bool measure, bool count_sweep)
{
    const long long fresh = fresh_energy_fx<NT>(sm, th);
    if (threadIdx.x == 0) {
        const double drift = fabs((double)(sm.st.E_fx - fresh) * kInvFx);
        if (drift > sm.st.max_drift) sm.st.max_drift = drift;
        sm.st.E_fx = fresh;
        if (count_sweep) {
            sm.st.sweep += 1u;
            sm.st.sweeps_done += 1ull;
        }
        if (measure) {
            const double dEm = (double)fresh * kInvFx - (sm.st.E_lo + 0.5 * sm.st.dE);
            sm.st.sum_dE += dEm;
            sm.st.sum_dE2 += dEm * dEm;
            sm.st.n_meas += 1;
        }
    }
    __syncthreads();
}

template <int NT, bool FAST>
__device__ void composite_sweep(Smem<NT> &sm, float *th, float a_f, uint32_t tag, int n_or,
                                int B, bool measure)
{
    full_pass<NT, FAST>(sm, th, 0, a_f, tag, B);
    for (int k = 0; k < n_or; ++k) full_pass<NT, FAST>(sm, th, 1, a_f, tag, B);
    end_of_sweep<NT>(sm, th, measure, true);
}

template <int NT, bool FAST>
__global__ void __launch_bounds__(NT) chain_kernel(ChainArgs args)
{
    __shared__ Smem<NT> sm;
    const int lat = args.order ? args.order[blockIdx.x] : (int)blockIdx.x;
    if (threadIdx.x == 0) {
        sm.st = args.lats[lat];
        sm.cap_cnt = 0ull;
        if (args.mode == kModePass && args.a_in) sm.st.a = args.a_in[lat];
        if (args.mode == kModeSweeps || args.mode == kModeRM) {
            if (args.a_in) sm.st.a = args.a_in[lat];
            sm.st.sum_dE = 0.0;
            sm.st.sum_dE2 = 0.0;
            sm.st.n_meas = 0;
        }
    }
    __syncthreads();
    float *th = args.theta + sm.st.off;

    if (args.mode == kModeResync) {
        const long long fresh = fresh_energy_fx<NT>(sm, th);
        if (threadIdx.x == 0) sm.st.E_fx = fresh;
    } else if (args.mode == kModePass) {
        full_pass<NT, FAST>(sm, th, args.pass_kind, (float)sm.st.a, kTagSweep, args.block,
                            args.class_mask);
    } else if (args.mode == kModeApproach) {
        int n = 0;
        for (;;) {
            const long long E = sm.st.E_fx;   // uniform after the last barrier
            if (dist_fx(E, sm.st.lo_fx, sm.st.hi_fx) == 0) break;
            if (n >= args.max_approach) {
                if (threadIdx.x == 0) sm.st.status = -3;   // LLR_ERR_WINDOW
                break;
            }
            const float a_f = (float)(E < sm.st.lo_fx ? -args.beta_up : -args.beta_dn);
            composite_sweep<NT, FAST>(sm, th, a_f, kTagApproach, args.n_or, args.block, false);
            ++n;
        }
        if (threadIdx.x == 0 && args.approach_sweeps) args.approach_sweeps[lat] = n;
    } else {
        const float a_f = (float)sm.st.a;
        const int total = args.n_therm + args.n_meas;
        for (int j = 0; j < total; ++j)
            composite_sweep<NT, FAST>(sm, th, a_f, kTagSweep, args.n_or, args.block,
                                      args.measure && j >= args.n_therm);
        if (threadIdx.x == 0) {
            if (args.mode == kModeRM) {
                const double mean = sm.st.n_meas > 0 ? sm.st.sum_dE / sm.st.n_meas : 0.0;
                const double a_new =
                    sm.st.a + 12.0 * mean / (sm.st.dE * sm.st.dE * (double)(args.rm_index + 1));
                if (!isfinite(a_new)) sm.st.status = -5;   // LLR_ERR_NUMERIC
                sm.st.a = a_new;
                if (args.a_out) args.a_out[lat] = a_new;
                if (args.mean_out) args.mean_out[lat] = mean;
            } else if (args.mean_out) {
                args.mean_out[lat] = sm.st.sum_dE;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        sm.st.caps += sm.cap_cnt;
        args.lats[lat] = sm.st;
    }
}

// ---------------------------------------------------------------------------
// Plain form: one lattice per launch, one launch per pass / resync / update.
// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(NT) plain_pass_kernel(ChainArgs args, int lat, int kind,
                                                        float a_f)
{
    __shared__ Smem<NT> sm;
    if (threadIdx.x == 0) {
        sm.st = args.lats[lat];
        sm.cap_cnt = 0ull;
    }
    __syncthreads();
    float *th = args.theta + sm.st.off;
    full_pass<NT, true>(sm, th, kind, a_f, kTagSweep, args.block);
    if (threadIdx.x == 0) {
        sm.st.caps += sm.cap_cnt;
        args.lats[lat] = sm.st;
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) plain_finish_kernel(ChainArgs args, int lat, int measure)
{
    __shared__ Smem<NT> sm;
    if (threadIdx.x == 0) sm.st = args.lats[lat];
    __syncthreads();
    end_of_sweep<NT>(sm, args.theta + sm.st.off, measure != 0, true);
    if (threadIdx.x == 0) args.lats[lat] = sm.st;
}

__global__ void plain_begin_kernel(ChainArgs args, int lat)
{
    LatState &st = args.lats[lat];
    if (args.a_in) st.a = args.a_in[lat];
    st.sum_dE = 0.0;
    st.sum_dE2 = 0.0;
    st.n_meas = 0;
}

__global__ void plain_update_kernel(ChainArgs args, int lat)
{
    LatState &st = args.lats[lat];
    const double mean = st.n_meas > 0 ? st.sum_dE / st.n_meas : 0.0;
    const double a_new = st.a + 12.0 * mean / (st.dE * st.dE * (double)(args.rm_index + 1));
    if (!isfinite(a_new)) st.status = -5;
    st.a = a_new;
    if (args.a_out) args.a_out[lat] = a_new;
    if (args.mean_out) args.mean_out[lat] = mean;
}

// ---------------------------------------------------------------------------
// Hot start: theta = -pi + 2 pi u (Haar measure), u from Philox with counter
// (link, 0, init tag, 0); computed in FP64 and rounded once to float.
// ---------------------------------------------------------------------------
__global__ void hot_start_kernel(LatState *lats, float *theta)
{
    const LatState st = lats[blockIdx.y];
    const int V = 2 * st.half;
    const int n = 4 * V;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const int mu = l / V, s = l - mu * V;
        const int L = st.L;
        const int x0 = s % L, x1 = (s / L) % L, x2 = (s / (L * L)) % L, x3 = s / (L * L * L);
        const int p = (x0 + x1 + x2 + x3) & 1;
        const U4 w = philox4x32_10((uint32_t)l, 0u, kTagInit, 0u, st.key0, st.key1);
        const double u = (double)((w.x >> 9) * 2u + 1u) * (1.0 / 16777216.0);
        const double t = __dadd_rn(-3.14159265358979323846, __dmul_rn(6.28318530717958647692, u));
        theta[st.off + (size_t)(2 * mu + p) * st.half + (s >> 1)] = (float)t;
    }
}

// FP64 fresh energy: plaquette angle and cos in double, warp-shuffle FP64
// reduction.  One CTA per lattice.
__global__ void __launch_bounds__(256) energy_fp64_kernel(const LatState *lats,
                                                          const float *theta, double *E_out)
{
    __shared__ double red[8];
    const LatState st = lats[blockIdx.x];
    const float *th = theta + st.off;
    const int L = st.L, half = st.half, V = 2 * half;
    const int stv[4] = {1, L, L * L, L * L * L};
    double acc = 0.0;
    for (int s = threadIdx.x; s < V; s += blockDim.x) {
        int x[4];
        x[0] = s % L;
        x[1] = (s / L) % L;
        x[2] = (s / (L * L)) % L;
        x[3] = s / (L * L * L);
        const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
        double t[4];
        int sp[4];
        for (int mu = 0; mu < 4; ++mu) {
            t[mu] = (double)th[(2 * mu + p) * half + (s >> 1)];
            sp[mu] = s + ((x[mu] == L - 1) ? -(L - 1) * stv[mu] : stv[mu]);
        }
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                const double b = (double)th[(2 * nu + (p ^ 1)) * half + (sp[mu] >> 1)];
                const double c = (double)th[(2 * mu + (p ^ 1)) * half + (sp[nu] >> 1)];
                acc += cos(((t[mu] + b) - c) - t[nu]);
            }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        E_out[blockIdx.x] = tot;
    }
}

__global__ void set_energy_kernel(LatState *lat, const double *E)
{
    lat->E_fx = __double2ll_rn(*E * kFx);
}

__global__ void to_canonical_kernel(const LatState *lat, const float *theta, float *out, int n)
{
    const LatState st = *lat;
    const int V = 2 * st.half, L = st.L;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const int mu = l / V, s = l - mu * V;
        const int p = (s % L + (s / L) % L + (s / (L * L)) % L + s / (L * L * L)) & 1;
        out[l] = theta[st.off + (size_t)(2 * mu + p) * st.half + (s >> 1)];
    }
}

__global__ void from_canonical_kernel(const LatState *lat, float *theta, const float *in, int n)
{
    const LatState st = *lat;
    const int V = 2 * st.half, L = st.L;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        const int mu = l / V, s = l - mu * V;
        const int p = (s % L + (s / L) % L + (s / (L * L)) % L + s / (L * L * L)) & 1;
        theta[st.off + (size_t)(2 * mu + p) * st.half + (s >> 1)] = in[l];
    }
}

template <int NT, bool FAST>
cudaError_t launch_chain_t(const ChainArgs &a, cudaStream_t s)
{
    chain_kernel<NT, FAST><<<a.n_lat, NT, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_chain(const ChainArgs &a, int threads, bool fast_math, cudaStream_t s)
{
    if (a.n_lat <= 0) return cudaSuccess;
    if (threads == 128) return fast_math ? launch_chain_t<128, true>(a, s) : launch_chain_t<128, false>(a, s);
    if (threads == 512) return fast_math ? launch_chain_t<512, true>(a, s) : launch_chain_t<512, false>(a, s);
    return fast_math ? launch_chain_t<256, true>(a, s) : launch_chain_t<256, false>(a, s);
}

cudaError_t launch_plain_begin(const ChainArgs &a, int lattice, cudaStream_t s)
{
    plain_begin_kernel<<<1, 1, 0, s>>>(a, lattice);
    return cudaGetLastError();
}

cudaError_t launch_plain_pass(const ChainArgs &a, int lattice, int kind, double a_val,
                              cudaStream_t s)
{
    plain_pass_kernel<256><<<1, 256, 0, s>>>(a, lattice, kind, (float)a_val);
    return cudaGetLastError();
}

cudaError_t launch_plain_finish(const ChainArgs &a, int lattice, int measure_this,
                                cudaStream_t s)
{
    plain_finish_kernel<256><<<1, 256, 0, s>>>(a, lattice, measure_this);
    return cudaGetLastError();
}

cudaError_t launch_plain_update(const ChainArgs &a, int lattice, cudaStream_t s)
{
    plain_update_kernel<<<1, 1, 0, s>>>(a, lattice);
    return cudaGetLastError();
}

cudaError_t launch_hot_start(LatState *lats, float *theta, int n_lat, int max_half,
                             cudaStream_t s)
{
    if (n_lat <= 0) return cudaSuccess;
    const int n = 8 * max_half;
    dim3 grid((unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), (unsigned)n_lat);
    hot_start_kernel<<<grid, 256, 0, s>>>(lats, theta);
    return cudaGetLastError();
}

cudaError_t launch_energy_fp64(const LatState *lats, const float *theta, int n_lat,
                               double *E_out, cudaStream_t s)
{
    if (n_lat <= 0) return cudaSuccess;
    energy_fp64_kernel<<<n_lat, 256, 0, s>>>(lats, theta, E_out);
    return cudaGetLastError();
}

cudaError_t launch_set_energy(LatState *lat_dev, const double *E_dev, cudaStream_t s)
{
    set_energy_kernel<<<1, 1, 0, s>>>(lat_dev, E_dev);
    return cudaGetLastError();
}

cudaError_t launch_to_canonical(const LatState *lat_dev, const float *theta, float *out,
                                int n_links, cudaStream_t s)
{
    to_canonical_kernel<<<(n_links + 255) / 256, 256, 0, s>>>(lat_dev, theta, out, n_links);
    return cudaGetLastError();
}

cudaError_t launch_from_canonical(const LatState *lat_dev, float *theta, const float *in,
                                  int n_links, cudaStream_t s)
{
    from_canonical_kernel<<<(n_links + 255) / 256, 256, 0, s>>>(lat_dev, theta, in, n_links);
    return cudaGetLastError();
}

}  // namespace llr
