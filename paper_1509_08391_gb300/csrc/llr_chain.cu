// llr_chain.cu -- the window-restricted Monte Carlo of 4-D compact U(1) on
// sm_103a: checkerboard staple sums, heat-bath and overrelaxation proposals,
// the sequential window-accept scan, the fresh energy and the Robbins-Monro
// update, for a batch of independent (interval, replica) lattices.
//
// Paper: Langfeld, Lucini, Pellegrini, Rago (arXiv:1509.08391).
//   Sec. 3.1      action E = sum_P cos(theta_P), plaquette angle
//                 theta_munu(x) = theta_mu(x) + theta_nu(x+mu) - theta_mu(x+nu) - theta_nu(x)
//   eqs. (2.13)-(2.16) weight exp(-a E) on the closed window [E_lo, E_lo + dE],
//                 dE_meas = E - E_lo - dE/2
//   Algorithm 1   n_therm + n_meas sweeps, measure after n_therm
//   eq. (2.30)      a <- a + 12 <<dE>> / (dE^2 (n + 1))
//
// Design
//   * Links are float32 angles, SoA by (direction, site parity), sites of a
//     parity in lexicographic order: theta[off + (2 mu + p) * V/2 + s/2].
//   * A heat-bath pass runs class by class over the whole lattice (one
//     pipeline drain per class); an overrelaxation pass is slab-major: for
//     each x3 slab, all 8 checkerboard classes of that slab in order, so a
//     slab's neighbourhood is reused from L2 by the 8 classes instead of each
//     class streaming the whole lattice.
//   * One persistent kernel.  Work items are (composite sweep j, lattice);
//     a CTA takes the next item from an atomic counter, waits (bounded) until
//     sweep j-1 of that lattice is done, and owns the lattice for that sweep.
//     Items run sweep-major, so uneven lattice sizes balance across SMs.
//   * In a heat-bath pass the warps are specialised: producer warps build
//     the six staples of one link per thread from 18 neighbour angles, draw
//     the von Mises proposal (Best & Fisher 1979), evaluate its dE from the
//     stored new angle exactly as the old local energy is evaluated, convert
//     dE to int64 fixed point (2^-32) and form warp prefix sums; a consumer
//     warp walks the chunks in link order and decides each block of B links
//     with the restricted Metropolis rule dist(E + dE_block) <= dist(E),
//     using a ballot to find the first rejected block among 32
//     speculatively accepted ones, and publishes an accept mask per group;
//     the producers write the accepted angles.  Chunks pass through a
//     4-stage shared memory ring guarded by named barriers, so proposals for
//     later chunks overlap with the scan of earlier ones.
//   * The multicanonical pass (Sec. 2.6) has the same producers at a fixed
//     proposal slope; its consumer replaces the window rule by a
//     Metropolis-Hastings test for the weight 1/rho~ in the same
//     speculative scan.
//   * Overrelaxation (theta' = -theta - 2 alpha) conserves E exactly, so its
//     passes skip the scan: every thread reflects links (neighbours read with
//     plain loads) and writes them directly.
//   * The per-class update, energy and update functions are not inlined, so
//     every program (batched sweeps, single passes, the plain form) runs the
//     same machine code and gives bit-identical results.
//   * After 1 + n_or passes the CTA sums the 6V plaquettes (float32 angles
//     summed exactly as hi + lo, cosf, fixed-point accumulation) and
//     resynchronises the tracked energy.
#include <cstdio>

#include "llr_internal.h"

namespace llr {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStages = 4;

// ---------------------------------------------------------------------------
// Best & Fisher (1979) von Mises sampler, density ~ exp(kappa cos X).
// tau = 1 + sqrt(1 + 4 k^2), rho = (tau - sqrt(2 tau)) / (2 k) (rewritten
// without cancellation), r = (1 + rho^2) / (2 rho).  Attempt t uses Philox
// call t/2 (counter word 3), words 0-1 (t even) or 2-3 (t odd) as u1, u2,
// and the lowest bit of the first of them as the sign of X:
// z = cos(pi u1), f = (1 + r z) / (r + z), c = k (r - f); accept if
// c (2 - c) > u2 or ln(c / u2) + 1 - c >= 0 (evaluated as
// log2 c - log2 u2 >= (c - 1) / ln 2).  The accept test runs on fast
// hardware approximations (it only decides which attempt is taken); the
// accepted variate is then evaluated without cancellation as (cos X, sin X),
// X = +-acos f: with sh, ch = sin, cos(pi u1 / 2) (hardware sine/cosine,
// absolute error ~5e-7 on [0, pi/2]), z = ch^2 - sh^2 and
//   1 - f = (r - 1) 2 sh^2 / (r + z)   (f >= 0),   1 + f = (r + 1) 2 ch^2 / (r + z)   (f < 0),
// so w = 1 -+ f has no cancellation, cos X = +-(1 - w) and
// |sin X| = sqrt(w (2 - w)) keep the angle's absolute accuracy near X = 0
// and X = pi.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool von_mises(float kappa, uint32_t c0, uint32_t c1, uint32_t c2,
                                          uint32_t k0, uint32_t k1, float &cX, float &sX)
{
    if (fabsf(kappa) < 1e-6f) {
        const U4 w = philox4x32_10(c0, c1, c2, 0u, k0, k1);
        const float t = 2.0f * u01(w.x) - 1.0f;   // X = pi t
        sincospif(t, &sX, &cX);
        return true;
    }
    const float k = fabsf(kappa);
    const float sq = sqrt_fast(fmaf(4.0f * k, k, 1.0f));
    const float tau = 1.0f + sq;
    const float rho = __fdividef(2.0f * k * tau, (sq + 1.0f) * (tau + sqrt_fast(2.0f * tau)));
    const float r = __fdividef(1.0f + rho * rho, 2.0f * rho);
    const float omr = 1.0f - rho;
    const float rm1 = __fdividef(omr * omr, 2.0f * rho);   // r - 1
    // find the first accepted attempt (cheap test only, so lanes that accept
    // at different attempts diverge over as little code as possible) ...
    bool found = false;
    uint32_t w_acc = 0u;
    for (int pair = 0; pair < kSamplerMaxAttempts / 2 && !found; ++pair) {
        const U4 w = philox4x32_10(c0, c1, c2, (uint32_t)pair, k0, k1);
#pragma unroll
        for (int half_ = 0; half_ < 2; ++half_) {
            const uint32_t wa = half_ ? w.z : w.x, wb = half_ ? w.w : w.y;
            const float u1 = u01(wa), u2 = u01(wb);
            const float z = __cosf(kPi * u1);
            const float f = __fdividef(1.0f + r * z, r + z);
            const float c = k * (rm1 + (1.0f - f));
            // second test ln(c / u2) + 1 - c >= 0, in base 2
            if (!found && (c * (2.0f - c) - u2 > 0.0f ||
                           __log2f(c) - __log2f(u2) >= (c - 1.0f) * 1.4426950408889634f)) {
                found = true;
                w_acc = wa;
            }
        }
    }
    if (!found) return false;
    // ... then evaluate the accepted variate once, without cancellation
    const float u1 = u01(w_acc);
    float sh, ch;
    __sincosf(0.5f * kPi * u1, &sh, &ch);
    const float z = (ch - sh) * (ch + sh);
    const float den = r + z;
    const bool pos = 1.0f + r * z >= 0.0f;                   // f >= 0
    const float w = __fdividef(pos ? rm1 * 2.0f * sh * sh : (r + 1.0f) * 2.0f * ch * ch, den);
    const float s = sqrt_fast(w * (2.0f - w));
    const float c = pos ? 1.0f - w : w - 1.0f;
    const bool neg_x = !(w_acc & 1u);                        // X = -acos f
    const bool flip = kappa < 0.0f;                          // X -> X + pi
    cX = flip ? -c : c;
    sX = (neg_x != flip) ? -s : s;
    return true;
}

template <bool FAST>
__device__ __forceinline__ void sin_cos(float x, float *s, float *c)
{
    if (FAST)
        __sincosf(x, s, c);
    else
        sincosf(x, s, c);
}

// arg(x + i y): the polynomial arctangent with fast math, the library's
// atan2f without.
template <bool FAST>
__device__ __forceinline__ float arg(float y, float x)
{
    return FAST ? arg_fast(y, x) : atan2f(y, x);
}

// Coordinates of the h-th site of parity p (lexicographic, x0 fastest).
__device__ __forceinline__ int decode_half(int h, int p, int L, uint32_t magic, int x[4])
{
    const int n = 2 * h;
    const int q = (int)__umulhi((uint32_t)n, magic);
    const int x0e = n - q * L;
    const int q2 = (int)__umulhi((uint32_t)q, magic);
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
//
// In a heat-bath pass the 18 neighbour angles are staged through shared
// memory: staple_fetch issues one 4-byte asynchronous copy (cp.async, cached
// in L1) per angle into the calling thread's column of a stage buffer, and
// staple_from sums the staples from it once the copies have landed, so a
// producer's loads for its next link overlap the sampling of the current one.  A thread only reads what it copied
// itself, so cp.async.wait_group is the only synchronisation.  The copies
// read through L1 like plain loads: other classes of this lattice were
// written earlier in the same launch (same CTA, or another CTA before the
// acquire of the lattice's done counter).
constexpr int kStaged = 18;   // angles per link in a stage column

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage the neighbour angles of link theta_MU(x) (site s, parity p) into
// col[k * stride], k = 6 j + (a1, a2, a3, b1, b2, b3) for the j-th nu != MU.
template <int MU>
__device__ __forceinline__ void staple_fetch(const float *th, int half, int L, const int x[4],
                                             int s, int p, float *col, int stride)
{
    const int st[4] = {1, L, L * L, L * L * L};
    const int dmu = (x[MU] == L - 1) ? -(L - 1) * st[MU] : st[MU];
    const int spmu = s + dmu;
    const int q = p ^ 1;
    const float *thmu_q = th + (2 * MU + q) * half;
    int j = 0;
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
        float *c = col + 6 * j * stride;
        cp_async4(c + 0 * stride, thnu_q + (spmu >> 1));      // theta_nu(x+mu)
        cp_async4(c + 1 * stride, thmu_q + (spnu >> 1));      // theta_mu(x+nu)
        cp_async4(c + 2 * stride, thnu_p + (s >> 1));         // theta_nu(x)
        cp_async4(c + 3 * stride, thnu_p + (smnu_pmu >> 1));  // theta_nu(x-nu+mu)
        cp_async4(c + 4 * stride, thmu_q + (smnu >> 1));      // theta_mu(x-nu)
        cp_async4(c + 5 * stride, thnu_q + (smnu >> 1));      // theta_nu(x-nu)
        ++j;
    }
}

template <bool FAST>
__device__ __forceinline__ void staple_from(const float *col, int stride, float &Sr, float &Si)
{
    Sr = 0.0f;
    Si = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float *c = col + 6 * j * stride;
        const float pf = c[0] - c[stride] - c[2 * stride];
        const float pb = c[5 * stride] - c[3 * stride] - c[4 * stride];
        float sf, cf, sb, cb;
        sin_cos<FAST>(pf, &sf, &cf);
        sin_cos<FAST>(pb, &sb, &cb);
        Sr += cf + cb;
        Si += sf + sb;
    }
}

// The stage buffer (dynamic shared memory): two columns sets of kStaged x NT
// floats, so the copies for a thread's next link land while it works on the
// current one.
extern __shared__ __align__(16) float g_stage_buf[];

template <int NT>
__device__ __forceinline__ float *stage_col(int buf)
{
    return g_stage_buf + buf * kStaged * NT + threadIdx.x;
}

// Named barriers 1..8 (0 is __syncthreads): stage s is full (1 + s) / empty (5 + s).
__device__ __forceinline__ void bar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <int NWP>
struct Stage {
    float thn[NWP * 32];
    long long P[NWP * 32];   // warp-inclusive prefix sums of dE (fixed point)
    unsigned endmask[NWP];
    unsigned accmask[NWP];   // written by the consumer: accepted block ends
};

template <int NWP>
struct Smem {
    LatState st;
    Stage<NWP> stage[kStages];
    long long red[NWP + 1];
    unsigned long long acc_cnt;
    unsigned long long cap_cnt;
    int item_lat, item_j, item_state;
    int cw;     // the consumer warp of a heat-bath pass
    int ring;   // stages of the ring in use (a power of two <= kStages)
};

// Producer side of one heat-bath class (MU, p): proposals and warp prefix
// sums, chunk by chunk, into the stage ring (slope a_f, Philox tag `tag`).
// When a slot comes back from the consumer (and for the last chunks at the
// end of the class) each producer writes its link's proposal if the
// consumer accepted the block it belongs to.
template <int MU, int NWP, bool FAST>
__device__ __noinline__ void produce_class(Smem<NWP> &sm, float *th, int p, float a_f,
                                           uint32_t tag, int B, int h0, int count, int nchunk,
                                           int D)
{
    constexpr int NT = (NWP + 1) * 32, CH = NWP * 32;
    // producer rank pt (0 .. CH-1) and producer warp pw: the warps other
    // than the consumer warp sm.cw, in order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int pw = w - (w > sm.cw ? 1 : 0), pt = pw * 32 + lane;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic, V = 2u * (uint32_t)half;
    const uint32_t k0 = sm.st.key0, k1 = sm.st.key1, sweep = sm.st.sweep;
    float *own = th + (2 * MU + p) * half;
    unsigned cnt = 0;
    // write back chunk c of a slot the consumer has released
    auto flush = [&](const Stage<NWP> &stg, int c) {
        const int lc = c * CH + pt;
        if (lc < count) {
            const int eb = __ffs(stg.endmask[pw] & ~((1u << lane) - 1u)) - 1;
            if ((stg.accmask[pw] >> eb) & 1u) {
                own[h0 + lc] = stg.thn[pt];
                ++cnt;
            }
        }
    };
    // prologue: stage the first chunk's neighbours
    bool valid_n = pt < count;
    int site_n = 0;
    float t0_n = 0.0f;
    if (valid_n) {
        int x[4];
        site_n = decode_half(h0 + pt, p, L, magic, x);
        staple_fetch<MU>(th, half, L, x, site_n, p, stage_col<NT>(0), NT);
        t0_n = own[h0 + pt];
    }
    cp_async_commit();
    for (int ch = 0; ch < nchunk; ++ch) {
        const int s = ch & (D - 1);
        const int local = ch * CH + pt;
        const bool valid = valid_n;
        const int site = site_n;
        const float t0 = t0_n;
        // stage the next chunk's neighbours while this one is sampled
        {
            const int ln = local + CH;
            valid_n = ch + 1 < nchunk && ln < count;
            if (valid_n) {
                int x[4];
                site_n = decode_half(h0 + ln, p, L, magic, x);
                staple_fetch<MU>(th, half, L, x, site_n, p, stage_col<NT>((ch + 1) & 1), NT);
                t0_n = own[h0 + ln];
            }
            cp_async_commit();
        }
        if (ch >= D) {
            bar_sync(5 + s, NT);
            flush(sm.stage[s], ch - D);
        }
        cp_async_wait<1>();
        float thn = 0.0f;
        long long d = 0;
        if (valid) {
            float Sr, Si;
            staple_from<FAST>(stage_col<NT>(ch & 1), NT, Sr, Si);
            float so, co;
            sin_cos<FAST>(t0, &so, &co);
            const float e_old = co * Sr - so * Si;     // |S| cos(theta + alpha)
            const float Sabs = sqrt_fast(Sr * Sr + Si * Si);
            float cX, sX;
            const uint32_t link = (uint32_t)MU * V + (uint32_t)site;
            if (von_mises(-a_f * Sabs, link, sweep, tag, k0, k1, cX, sX)) {
                // theta' = X - alpha, alpha = arg S: e^{i theta'} = e^{iX} conj(S) / |S|
                thn = arg<FAST>(sX * Sr - cX * Si, cX * Sr + sX * Si);
                // dE of the angle actually stored, evaluated exactly like e_old
                // (same staple sum, same sine/cosine): the approximation errors
                // of one link's successive evaluations then cancel along its
                // chain of updates and leave only random noise.  Taking
                // |S| cos X instead carried a systematic -3.5e-8 per move (the
                // rounded atan2 and (cos X, sin X) are not exactly the angle
                // X - alpha), which drifted the running energy by -4.8e-4 per
                // heat-bath pass at L = 8 and shifted the window it enforces.
                float sn, cn;
                sin_cos<FAST>(thn, &sn, &cn);
                d = to_fx((cn * Sr - sn * Si) - e_old);
            } else {
                thn = t0;
                atomicAdd(&sm.cap_cnt, 1ull);
            }
        }
        long long P = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(kFull, P, o);
            if (lane >= o) P += y;
        }
        const bool isend = valid && (((lane & (B - 1)) == B - 1) || local == count - 1);
        const unsigned em = __ballot_sync(kFull, isend);
        Stage<NWP> &stg = sm.stage[s];
        stg.thn[pt] = thn;
        stg.P[pt] = P;
        if (lane == 0) stg.endmask[pw] = em;
        bar_arrive(1 + s, NT);
    }
    for (int c = nchunk > D ? nchunk - D : 0; c < nchunk; ++c) {
        const int s = c & (D - 1);
        bar_sync(5 + s, NT);
        flush(sm.stage[s], c);
    }
    cp_async_wait<0>();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
    if (lane == 0) atomicAdd(&sm.acc_cnt, (unsigned long long)cnt);
}

// Neighbour angles of link theta_MU(x) (site s, parity p) loaded straight into
// registers v[18], in the order of staple_fetch.
template <int MU>
__device__ __forceinline__ void staple_load(const float *th, int half, int L, const int x[4],
                                            int s, int p, float v[18])
{
    const int st[4] = {1, L, L * L, L * L * L};
    const int dmu = (x[MU] == L - 1) ? -(L - 1) * st[MU] : st[MU];
    const int spmu = s + dmu;
    const int q = p ^ 1;
    const float *thmu_q = th + (2 * MU + q) * half;
    int j = 0;
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
        v[6 * j + 0] = thnu_q[spmu >> 1];
        v[6 * j + 1] = thmu_q[spnu >> 1];
        v[6 * j + 2] = thnu_p[s >> 1];
        v[6 * j + 3] = thnu_p[smnu_pmu >> 1];
        v[6 * j + 4] = thmu_q[smnu >> 1];
        v[6 * j + 5] = thnu_q[smnu >> 1];
        ++j;
    }
}

// Staple sum of one link from its 18 neighbour angles, formed exactly as in
// staple_from.
template <bool FAST>
__device__ __forceinline__ void staple_sum_regs(const float v[18], float &Sr, float &Si)
{
    Sr = 0.0f;
    Si = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float pf = v[6 * j] - v[6 * j + 1] - v[6 * j + 2];
        const float pb = v[6 * j + 5] - v[6 * j + 3] - v[6 * j + 4];
        float sf, cf, sb, cb;
        sin_cos<FAST>(pf, &sf, &cf);
        sin_cos<FAST>(pb, &sb, &cb);
        Sr += cf + cb;
        Si += sf + sb;
    }
}

// Overrelaxation and the window.  A reflection keeps the local energy
// |S| cos(theta + alpha) exactly; a move changes E only through float32
// rounding (the reflection axis alpha carries the staple sum's error, ~1e-6 /
// |S|, the stored angle its rounding), and its float32 dE estimate is as
// uncertain as that change.  So the running energy is not changed by
// overrelaxation, and a block of a group is taken iff E -- the running energy
// at the start of the group -- lies outside the window, or E + dE_block lies
// inside it (reading R19).  Every |dE| is below 2^-14 (a move whose float32
// estimate exceeds that is refused, a guard never expected to act), so while
// E is outside the window, or inside and farther than B * 2^-14 from both
// edges, every move is taken without evaluating a dE.
constexpr float kOrDeltaMax = 6.103515625e-05f;   // 2^-14
constexpr long long kOrDeltaMaxFx = 1ll << 18;
constexpr int kOrRefused = (int)0x80000000;

// theta' = -theta - 2 alpha of link theta_MU at half-site h of parity p, with
// alpha = arg S (S from the 18 neighbour angles, plain loads); optionally the
// float32 dE estimate in fixed point, evaluated like the heat-bath's: the local
// energy Re(e^{i theta} S) at the stored new angle minus at the old one, same
// staple sum, same sine/cosine (dfx = kOrRefused beyond the guard).
template <int MU, bool FAST, bool WITH_DE>
__device__ __forceinline__ float overrelax_link(const float *th, const float *own, int half, int L,
                                                uint32_t magic, int p, int h, int &dfx)
{
    float va[18];
    int x[4];
    const int site = decode_half(h, p, L, magic, x);
    staple_load<MU>(th, half, L, x, site, p, va);
    const float t0 = own[h];
    float Sr, Si;
    staple_sum_regs<FAST>(va, Sr, Si);
    const float tn = wrap_angle(-t0 - 2.0f * arg<FAST>(Si, Sr));
    if (WITH_DE) {
        float sn, cn, so, co;
        sin_cos<FAST>(tn, &sn, &cn);
        sin_cos<FAST>(t0, &so, &co);
        const float d = (cn * Sr - sn * Si) - (co * Sr - so * Si);
        dfx = fabsf(d) <= kOrDeltaMax ? __float2int_rn(d * 4294967296.0f) : kOrRefused;
    }
    return tn;
}

// One overrelaxation group (the links of class (MU, p) with half-site index
// in [h0, h0 + count)) whose running energy E lies outside the window, or
// inside and farther than B * 2^-14 from both edges: every move is taken by
// the window rule, so no dE is needed.  Every thread reflects its links and
// writes them directly.  The neighbours are plain loads: within a slab they
// mostly hit L1/L2, and with no consumer to feed, the loads of many warps
// hide each other.
template <int MU, int NWP, bool FAST>
__device__ __noinline__ void overrelax_class(Smem<NWP> &sm, float *th, int p, int h0, int count)
{
    constexpr int NT = (NWP + 1) * 32;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic;
    float *own = th + (2 * MU + p) * half;
    for (int local = threadIdx.x; local < count; local += NT) {
        int dfx;
        own[h0 + local] =
            overrelax_link<MU, FAST, false>(th, own, half, L, magic, p, h0 + local, dfx);
    }
}

// Heat-bath window decisions of one 32-link group in link order, by the
// calling warp.  Lane k holds Pk, the inclusive prefix sum of dE over the
// group's links 0..k; em marks the lanes that end a block (blocks of B links
// start at multiples of B).  A block is taken iff dist(E + dE_block) <=
// dist(E), dist the distance from the closed window (inside the window: iff
// the energy after the block is inside).  Returns the mask of taken block
// ends and advances E.
__device__ __forceinline__ unsigned window_scan_group(long long Pk, unsigned em, int B,
                                                      long long &E, long long lo, long long hi)
{
    const int lane = threadIdx.x & 31;
    unsigned rem = em, acc = 0u;
    // the sum of the block ending at this lane
    const int bstart = lane & ~(B - 1);
    const long long Pprev = __shfl_sync(kFull, Pk, bstart > 0 ? bstart - 1 : 0);
    const long long bk = Pk - (bstart > 0 ? Pprev : 0ll);
    if (em != 0u && E >= lo && E <= hi) {
        // Inside the window (the usual case, and E stays inside): a block is
        // taken iff lo - E <= Pk - R <= hi - E, R the sum of the blocks
        // refused so far.  Keep the bounds rlo = lo - E + R, rhi = hi - E + R;
        // a refusal at j adds its block sum bj.
        long long rlo = lo - E, rhi = hi - E;
        while (rem) {
            const bool mine = (rem >> lane) & 1u;
            const bool viol = mine && (Pk < rlo || Pk > rhi);
            const unsigned vm = __ballot_sync(kFull, viol);
            if (vm == 0u) {
                acc |= rem;
                break;
            }
            const int j = __ffs(vm) - 1;
            acc |= rem & ((1u << j) - 1u);
            const long long bj = __shfl_sync(kFull, bk, j);
            rlo += bj;
            rhi += bj;
            rem &= ~((2u << j) - 1u);
        }
        // E after the group = E + P_last - R = lo + P_last - rlo
        E = lo + __shfl_sync(kFull, Pk, 31 - __clz(em)) - rlo;
    } else {
        // Outside the window: every remaining block is decided as if the
        // earlier ones were taken; the first refusal (one ballot) fixes the
        // blocks before it, its dE is dropped and the rest is decided again.
        long long base = 0;
        while (rem) {
            const long long Ea = E + (Pk - base);
            const long long Eb = Ea - bk;
            const bool mine = (rem >> lane) & 1u;
            const bool ok = dist_fx(Ea, lo, hi) <= dist_fx(Eb, lo, hi);
            const unsigned vm = __ballot_sync(kFull, mine && !ok);
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
                E += (Pj - bj) - base;   // energy before the refused block
                base = Pj;               // skip its contribution
                rem &= ~((2u << j) - 1u);
            }
        }
    }
    return acc;
}

// One overrelaxation group whose running energy E is inside the window and
// within B * 2^-14 of an edge: every thread forms its links' moves and float32
// dE estimates;
// the blocks of B links (starting at the group's first link; a block lies in
// one warp) sum their dE with shuffles, and a block is taken iff E lies
// outside the window or E + dE_block inside it.  Decisions are independent of
// one another (E does not move), so no barrier is needed.  Returns the number
// of moves this thread took.
template <int MU, int NWP, bool FAST>
__device__ __noinline__ int overrelax_class_near(Smem<NWP> &sm, float *th, int p, int h0,
                                                 int count, int B, long long E)
{
    constexpr int NT = (NWP + 1) * 32;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic;
    const long long lo = sm.st.lo_fx, hi = sm.st.hi_fx;
    const bool outside = E < lo || E > hi;
    float *own = th + (2 * MU + p) * half;
    int taken = 0;
    for (int c0 = 0; c0 < count; c0 += NT) {
        const int local = c0 + threadIdx.x;
        const bool valid = local < count;
        int dfx = 0;
        float tn = 0.0f;
        bool ok = false;
        if (valid) {
            tn = overrelax_link<MU, FAST, true>(th, own, half, L, magic, p, h0 + local, dfx);
            ok = dfx != kOrRefused;
            if (!ok) dfx = 0;
        }
        long long d = dfx;   // the block's dE (lanes of one block are an aligned segment)
        for (int o = 1; o < B; o <<= 1) d += __shfl_xor_sync(kFull, d, o);
        const long long Eb = E + d;
        if (valid && ok && (outside || (Eb >= lo && Eb <= hi))) {
            own[h0 + local] = tn;
            ++taken;
        }
    }
    return taken;
}

// Consumer side: sequential Metropolis accept of the chunk's blocks in link
// order; publishes the accepted block ends of each group (the producers
// write the angles).  Runs in the last warp.
template <int NWP>
__device__ __noinline__ void consume_class(Smem<NWP> &sm, int B, int nchunk, int D)
{
    constexpr int NT = (NWP + 1) * 32;
    const int lane = threadIdx.x & 31;
    long long E = sm.st.E_fx;
    const long long lo = sm.st.lo_fx, hi = sm.st.hi_fx;
    for (int ch = 0; ch < nchunk; ++ch) {
        const int s = ch & (D - 1);
        bar_sync(1 + s, NT);
        Stage<NWP> &stg = sm.stage[s];
        for (int g = 0; g < NWP; ++g) {
            const unsigned acc =
                window_scan_group(stg.P[g * 32 + lane], stg.endmask[g], B, E, lo, hi);
            if (lane == 0) stg.accmask[g] = acc;
        }
        bar_arrive(5 + s, NT);
    }
    if (lane == 0) sm.st.E_fx = E;
}

// ln rho~ of the multicanonical weight at the fixed-point energy E: the
// piecewise-linear function of eq. (2.10) on the table's intervals,
// continued with the first / last slope beyond them (Sec. 2.6, eq. (2.50)).
__device__ __forceinline__ double muca_lnrho(const KernelArgs &a, long long E_fx)
{
    const double E = (double)E_fx * kInvFx;
    int k = (int)floor((E - a.muca_e0) / a.muca_de);
    k = k < 0 ? 0 : (k > a.muca_n - 1 ? a.muca_n - 1 : k);
    return a.muca_lnr[k] + a.muca_a[k] * (E - (a.muca_e0 + (double)k * a.muca_de));
}

// Consumer side of a multicanonical heat-bath class (Sec. 2.6): the links
// of each 32-link group are taken in link order by Metropolis-Hastings for
// the weight 1/rho~ with the proposal at slope a0, i.e. with probability
// min(1, exp(a0 dE - (ln rho~(E + dE) - ln rho~(E)))), E the running energy
// before the link; the uniform comes from Philox counter (link, sweep, 12, 0).
// Speculatively every remaining link is decided as if all earlier ones were
// taken; the first refusal (one ballot) fixes the links before it, its dE is
// dropped and the rest is decided again.  Blocks of one link.
template <int NWP>
__device__ __noinline__ void consume_class_muca(Smem<NWP> &sm, int nchunk, int mu, int p,
                                                const KernelArgs &args, int D)
{
    constexpr int NT = (NWP + 1) * 32, CH = NWP * 32;
    const int lane = threadIdx.x & 31;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic, V = 2u * (uint32_t)half;
    const uint32_t k0 = sm.st.key0, k1 = sm.st.key1, sweep = sm.st.sweep;
    const double a0 = args.muca_a0;
    long long E = sm.st.E_fx;
    for (int ch = 0; ch < nchunk; ++ch) {
        const int s = ch & (D - 1);
        bar_sync(1 + s, NT);
        Stage<NWP> &stg = sm.stage[s];
        for (int g = 0; g < NWP; ++g) {
            const unsigned em = stg.endmask[g];
            unsigned rem = em, acc = 0u;
            const long long Pk = stg.P[g * 32 + lane];
            const long long Pprev = __shfl_up_sync(kFull, Pk, 1);
            const long long dk = lane > 0 ? Pk - Pprev : Pk;
            double u = 1.0;
            if ((em >> lane) & 1u) {
                int x[4];
                const int site = decode_half(ch * CH + g * 32 + lane, p, L, magic, x);
                const U4 w = philox4x32_10((uint32_t)mu * V + (uint32_t)site, sweep, kTagMuca, 0u,
                                           k0, k1);
                u = (double)u01(w.x);
            }
            long long R = 0;
            while (rem) {
                const bool mine = (rem >> lane) & 1u;
                bool refuse = false;
                if (mine) {
                    const long long Eb = E + (Pk - dk) - R;
                    const double xk =
                        a0 * ((double)dk * kInvFx) - (muca_lnrho(args, Eb + dk) - muca_lnrho(args, Eb));
                    refuse = !(u < exp(xk));
                }
                const unsigned vm = __ballot_sync(kFull, refuse);
                if (vm == 0u) {
                    acc |= rem;
                    break;
                }
                const int j = __ffs(vm) - 1;
                acc |= rem & ((1u << j) - 1u);
                R += __shfl_sync(kFull, dk, j);
                rem &= ~((2u << j) - 1u);
            }
            if (em != 0u) E += __shfl_sync(kFull, Pk, 31 - __clz(em)) - R;
            if (lane == 0) stg.accmask[g] = acc;
        }
        bar_arrive(5 + s, NT);
    }
    if (lane == 0) sm.st.E_fx = E;
}

// One pass over the selected classes (mu = 0..3, parity 0,1).  Heat-bath:
// class by class over the whole lattice.  Overrelaxation: slab by slab of the
// last coordinate (x3 = t, the h range [t S, (t+1) S) of every class array,
// S = L^3 / 2) and the classes within each slab, each group under the window
// rule of the running energy (windowed false: no window, every reflection
// is taken -- the multicanonical run).
template <int NWP, bool FAST>
__device__ void run_pass(Smem<NWP> &sm, float *th, int kind, float a_f, uint32_t tag, int B,
                         int class_mask, const KernelArgs *muca = nullptr, bool windowed = true)
{
    constexpr int NT = (NWP + 1) * 32, CH = NWP * 32;
    if (threadIdx.x == 0) sm.acc_cnt = 0ull;
    __syncthreads();
    const int half = sm.st.half, L = sm.st.L;
    const int D = sm.ring;   // stages of the producer/consumer ring in use: 1, 2 or 4
    if (kind == 1) {
        // Overrelaxation: slab by slab (x3), all classes within a slab, so the
        // neighbours a slab's staples read are still in L2 from the class before.
        const int S = half / L;
        const long long lo = windowed ? sm.st.lo_fx : -(1ll << 62);
        const long long hi = windowed ? sm.st.hi_fx : (1ll << 62);
        // a block's |dE| is below B 2^-14, so no block can be refused unless E
        // is inside the window and within that of an edge
        const long long bound = (long long)B * kOrDeltaMaxFx;
        const long long E = sm.st.E_fx;   // the running energy; overrelaxation leaves it
        const bool free_all = E < lo || E > hi || (E - bound >= lo && E + bound <= hi);
        int taken = 0;              // moves taken by this thread in near-edge groups
        unsigned long long n_free = 0;
#pragma unroll 1
        for (int t = 0; t < L; ++t) {
#pragma unroll 1
            for (int cls = 0; cls < 8; ++cls) {
                if (!((class_mask >> cls) & 1)) continue;
                const int p = cls & 1;
                if (free_all) {
                    switch (cls >> 1) {
                        case 0: overrelax_class<0, NWP, FAST>(sm, th, p, t * S, S); break;
                        case 1: overrelax_class<1, NWP, FAST>(sm, th, p, t * S, S); break;
                        case 2: overrelax_class<2, NWP, FAST>(sm, th, p, t * S, S); break;
                        default: overrelax_class<3, NWP, FAST>(sm, th, p, t * S, S); break;
                    }
                    n_free += (unsigned long long)S;
                } else {
                    switch (cls >> 1) {
                        case 0: taken += overrelax_class_near<0, NWP, FAST>(sm, th, p, t * S, S, B, E); break;
                        case 1: taken += overrelax_class_near<1, NWP, FAST>(sm, th, p, t * S, S, B, E); break;
                        case 2: taken += overrelax_class_near<2, NWP, FAST>(sm, th, p, t * S, S, B, E); break;
                        default: taken += overrelax_class_near<3, NWP, FAST>(sm, th, p, t * S, S, B, E); break;
                    }
                }
                __syncthreads();   // the next group reads the angles written here
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) taken += __shfl_down_sync(kFull, taken, o);
        if ((threadIdx.x & 31) == 0 && taken) atomicAdd(&sm.acc_cnt, (unsigned long long)taken);
        if (threadIdx.x == 0 && n_free) atomicAdd(&sm.acc_cnt, n_free);
        (void)NT;
    } else {
        // Heat-bath: one class at a time over the whole lattice, so the
        // producer/consumer pipeline drains once per class.
        const int nchunk = (half + CH - 1) / CH;
        const bool consumer = (threadIdx.x >> 5) == sm.cw;
#pragma unroll 1
        for (int cls = 0; cls < 8; ++cls) {
            if (!((class_mask >> cls) & 1)) continue;
            const int mu = cls >> 1, p = cls & 1;
            if (consumer) {
                if (kind == 2)
                    consume_class_muca<NWP>(sm, nchunk, mu, p, *muca, D);
                else
                    consume_class<NWP>(sm, B, nchunk, D);
            } else {
                switch (mu) {
                    case 0: produce_class<0, NWP, FAST>(sm, th, p, a_f, tag, B, 0, half, nchunk, D); break;
                    case 1: produce_class<1, NWP, FAST>(sm, th, p, a_f, tag, B, 0, half, nchunk, D); break;
                    case 2: produce_class<2, NWP, FAST>(sm, th, p, a_f, tag, B, 0, half, nchunk, D); break;
                    default: produce_class<3, NWP, FAST>(sm, th, p, a_f, tag, B, 0, half, nchunk, D); break;
                }
            }
            __syncthreads();   // the next class reads the angles written here
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long n =
            (unsigned long long)__popc(class_mask & 0xFF) * (unsigned long long)half;
        if (kind != 1) {
            sm.st.hb_acc += sm.acc_cnt;
            sm.st.hb_tot += n;
        } else {
            sm.st.or_acc += sm.acc_cnt;
            sm.st.or_tot += n;
        }
    }
    __syncthreads();
}

// cos(x) for x = hi + lo (|hi| <= 4 pi, |lo| tiny), accurate to about one
// ulp and without systematic error, for the fixed-point plaquette sums: a
// per-plaquette bias of 1e-9 would add up to ~1e-3 over the 960000
// plaquettes of an L = 20 lattice (the accurate sincosf showed a mean error of
// that order there), shifting the measured <<dE>>.
//   Reduction (Cody & Waite, "Software Manual for the Elementary Functions",
//   1980): k = nearest integer to hi 2/pi and x - k pi/2 = rh + rl with pi/2
//   split into P1 + P2 + P3 (P1, P2 of 20 significant bits, so k P1 and k P2
//   are exact for |k| <= 8): rh = hi - k P1 is exact and rl = lo - k P2 - k P3
//   is tiny.  Rounding x - k P2 to one float instead would repeat the same
//   rounding error for every angle of a binade (hi - k P1 lies on the float
//   grid), a bias of ~2e-10 per plaquette.
//   Evaluation: the Taylor series of cos and sin at rh in z = rh^2, truncated
//   where the next term is below 1e-15; the coefficients 1/4!, 1/3! and 1/5!
//   are carried as float pairs (their float rounding alone would bias the
//   result by up to 5e-9); then cos(rh + rl) = cos rh - rl sin rh and
//   sin(rh + rl) = sin rh + rl cos rh (plus the rl^2 terms), and
//   cos x = cos r, -sin r, -cos r, sin r for k = 0, 1, 2, 3 (mod 4).
__device__ __forceinline__ float cos_unbiased(float hi, float lo)
{
    const float k = rintf(hi * 0.636619747f);
    const float rh = fmaf(-k, 1.5707950592041016f, hi);
    float rl = fmaf(-k, 1.2675900507019833e-06f, lo);
    rl = fmaf(-k, 7.4435477313145038e-13f, rl);
    const float z = rh * rh;
    // cos rh = 1 - z/2 + z^2/4! - ... - z^7/14!
    float c = -1.147074536e-11f;
    c = fmaf(c, z, 2.087675588e-09f);
    c = fmaf(c, z, -2.755731998e-07f);
    c = fmaf(c, z, 2.480158764e-05f);
    c = fmaf(c, z, -1.388888923e-03f);
    c = fmaf(c, z, -1.241763470e-09f);   // 1/4! = 4.166666791e-02 - 1.241763470e-09
    c += 4.166666791e-02f;
    c = fmaf(c, z, -0.5f);
    c = fmaf(c, z, 1.0f);
    // sin rh = rh (1 - z/3! + z^2/5! - ... - z^7/15!)
    float t = -7.647163610e-13f;
    t = fmaf(t, z, 1.605904437e-10f);
    t = fmaf(t, z, -2.505210794e-08f);
    t = fmaf(t, z, 2.755731884e-06f);
    t = fmaf(t, z, -1.984127011e-04f);
    t = fmaf(t, z, -4.346172033e-10f);   // 1/5! = 8.333333768e-03 - 4.346172033e-10
    t += 8.333333768e-03f;
    t = fmaf(t, z, 4.967053879e-09f);    // 1/3! = 1.666666716e-01 - 4.967053879e-09
    t -= 1.666666716e-01f;
    t = rh * fmaf(t, z, 1.0f);
    // cos(rh + rl), sin(rh + rl) to second order in rl (|rl| <= 1e-5: the
    // dropped -rl^2/2 alone would bias cos by up to -5e-11); the small terms
    // are summed first, so the correction is not rounded away
    const float h = 0.5f * rl * rl;
    const float cr = c - fmaf(t, rl, c * h);
    const float sr = t + fmaf(c, rl, -t * h);
    const int q = (int)k & 3;
    const float v = (q & 1) ? sr : cr;
    return (q == 1 || q == 2) ? -v : v;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// cos of the plaquette angle a + b - c - d of four float angles: the angle is
// formed exactly as hi + lo and its cosine taken by cos_unbiased.
__device__ __forceinline__ float plaquette_cos(float a, float b, float c, float d)
{
    float s1, e1, s2, e2, hi, e3;
    two_sum(a, b, s1, e1);
    two_sum(c, d, s2, e2);
    two_sum(s1, -s2, hi, e3);
    const float lo = (e1 - e2) + e3;
    return cos_unbiased(hi, lo);
}

// Fresh energy of the CTA's lattice in fixed point: sum over the 6 V
// plaquettes, exact int64 accumulation and reduction.  Valid in thread 0.
template <int NWP>
__device__ __noinline__ long long fresh_energy_fx(Smem<NWP> &sm, const float *th)
{
    constexpr int NT = (NWP + 1) * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int L = sm.st.L, half = sm.st.half;
    const uint32_t magic = sm.st.magic;
    const int V = 2 * half;
    const int st[4] = {1, L, L * L, L * L * L};
    long long acc = 0;
    for (int s = tid; s < V; s += NT) {
        int x[4];
        const int q = (int)__umulhi((uint32_t)s, magic);
        x[0] = s - q * L;
        const int q2 = (int)__umulhi((uint32_t)q, magic);
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
            t[mu] = th[(2 * mu + p) * half + hs];
            sp[mu] = s + ((x[mu] == L - 1) ? -(L - 1) * st[mu] : st[mu]);
        }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu)
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                const float tnu_xmu = th[(2 * nu + (p ^ 1)) * half + (sp[mu] >> 1)];
                const float tmu_xnu = th[(2 * mu + (p ^ 1)) * half + (sp[nu] >> 1)];
                acc += to_fx(plaquette_cos(t[mu], tnu_xmu, tmu_xnu, t[nu]));
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o);
    if (lane == 0) sm.red[warp] = acc;
    __syncthreads();
    long long tot = 0;
    if (tid == 0)
        for (int w = 0; w < NWP + 1; ++w) tot += sm.red[w];
    __syncthreads();
    return tot;
}

// Resync after a composite sweep; thread 0 updates the state.
template <int NWP>
__device__ void end_of_sweep(Smem<NWP> &sm, const float *th, bool measure)
{
    const long long fresh = fresh_energy_fx<NWP>(sm, th);
    if (threadIdx.x == 0) {
        const double drift = fabs((double)(sm.st.E_fx - fresh) * kInvFx);
        if (drift > sm.st.max_drift) sm.st.max_drift = drift;
        sm.st.E_fx = fresh;
        sm.st.sweep += 1u;
        sm.st.sweeps_done += 1ull;
        if (measure) {
            const double dEm = (double)fresh * kInvFx - (sm.st.E_lo + 0.5 * sm.st.dE);
            sm.st.sum_dE += dEm;
            sm.st.sum_dE2 += dEm * dEm;
            sm.st.n_meas += 1;
        }
    }
    __syncthreads();
}

template <int NWP, bool FAST>
__device__ void composite_sweep(Smem<NWP> &sm, float *th, float a_f, uint32_t tag, int n_or,
                                int B, bool measure)
{
    run_pass<NWP, FAST>(sm, th, 0, a_f, tag, B, 0xFF);
    for (int k = 0; k < n_or; ++k) run_pass<NWP, FAST>(sm, th, 1, a_f, tag, B, 0xFF);
    end_of_sweep<NWP>(sm, th, measure);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Robbins-Monro update of the CTA's lattice (thread 0).
__device__ __noinline__ void rm_update(LatState &st, const KernelArgs &args, int lat)
{
    const int step = args.step_dev ? *args.step_dev : 0;
    const double mean = st.n_meas > 0 ? st.sum_dE / st.n_meas : 0.0;
    const double a_new =
        st.a + 12.0 * mean / (st.dE * st.dE * (double)(args.rm_index + step + 1));
    if (!isfinite(a_new)) st.status = -5;   // LLR_ERR_NUMERIC
    st.a = a_new;
    if (args.a_out) args.a_out[lat] = a_new;
    if (args.mean_out) args.mean_out[lat] = mean;
    if (args.hist) args.hist[(size_t)step * (size_t)args.n_lat + (size_t)lat] = a_new;
}

// Resident CTAs per SM the register budget is held to: 512 threads x 2 (64
// registers); 128 threads x 6, 160 threads x 5, 192 threads x 4 and 256
// threads x 3 (80 registers).
template <int NWP>
constexpr int min_ctas()
{
    return NWP == 3 ? 6 : NWP == 4 ? 5 : NWP == 5 ? 4 : NWP == 7 ? 3 : 2;
}

template <int NWP, bool FAST>
__global__ void __launch_bounds__((NWP + 1) * 32, min_ctas<NWP>()) llr_kernel(KernelArgs args)
{
    __shared__ Smem<NWP> sm;
    const int tid = threadIdx.x;
    const bool multi =
        args.program == kProgSweeps || args.program == kProgRM || args.program == kProgMuca;
    const int per_lat = multi ? args.n_therm + args.n_meas : 1;
    const unsigned n_items = (unsigned)args.n_lat * (unsigned)per_lat;
    unsigned *err = args.sync;
    unsigned *counter = args.sync + 1;
    unsigned *done = args.sync + 2;
    if (tid == 0) {
        sm.cw = NWP;   // the consumer warp of a heat-bath pass: the last
        sm.ring = (args.ring == 1 || args.ring == 2) ? args.ring : kStages;
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const unsigned i = atomicAdd(counter, 1u);
            int state = 0;
            if (i < n_items) {
                const int j = (int)(i / (unsigned)args.n_lat);
                const int slot = (int)(i % (unsigned)args.n_lat);
                state = 1;
                if (j > 0) {
                    // sweep j-1 of this lattice was dequeued earlier by a running
                    // CTA; wait for it, but never longer than wait_limit_ns.  Once
                    // any wait has run out (the error word is set; it stays set
                    // until the host reads it), an item that would wait skips at
                    // once: the sweep before it may never come.
                    const unsigned long long t0 = global_ns();
                    while (ld_acquire(done + slot) < (unsigned)j) {
                        if (ld_acquire(err) != 0u) {
                            state = 2;
                            break;
                        }
                        if (global_ns() - t0 > args.wait_limit_ns) {
                            atomicOr(err, 1u);
                            state = 2;
                            break;
                        }
                        __nanosleep(256);
                    }
                }
                sm.item_lat = slot;
                sm.item_j = j;
                if (state == 1) sm.st = args.lats[args.order ? args.order[slot] : slot];
            }
            sm.item_state = state;
            sm.cap_cnt = 0ull;
        }
        __syncthreads();
        const int state = sm.item_state;
        if (state == 0) break;
        if (state == 2) {
            __syncthreads();
            continue;   // timed out: leave this lattice alone, the host reads the error word
        }
        const int slot = sm.item_lat, j = sm.item_j;
        const int lat = args.order ? args.order[slot] : slot;
        float *th = args.theta + sm.st.off;

        switch (args.program) {
            case kProgSweeps:
            case kProgRM: {
                if (j == 0 && tid == 0) {
                    if (args.a_in) sm.st.a = args.a_in[lat];
                    sm.st.sum_dE = 0.0;
                    sm.st.sum_dE2 = 0.0;
                    sm.st.n_meas = 0;
                }
                __syncthreads();
                const float a_f = (float)sm.st.a;
                composite_sweep<NWP, FAST>(sm, th, a_f, kTagSweep, args.n_or, args.block,
                                           args.measure && j >= args.n_therm);
                if (j == per_lat - 1 && tid == 0) {
                    if (args.program == kProgRM)
                        rm_update(sm.st, args, lat);
                    else if (args.mean_out)
                        args.mean_out[lat] = sm.st.sum_dE;
                }
                break;
            }
            case kProgApproach: {
                int n = 0;
                for (;;) {
                    const long long E = sm.st.E_fx;   // uniform after the last barrier
                    if (dist_fx(E, sm.st.lo_fx, sm.st.hi_fx) == 0) break;
                    if (n >= args.max_approach) {
                        if (tid == 0) sm.st.status = -3;   // LLR_ERR_WINDOW
                        break;
                    }
                    const float a_f = (float)(E < sm.st.lo_fx ? -args.beta_up : -args.beta_dn);
                    composite_sweep<NWP, FAST>(sm, th, a_f, kTagApproach, args.n_or, args.block,
                                               false);
                    ++n;
                }
                if (tid == 0 && args.approach_sweeps) args.approach_sweeps[lat] = n;
                break;
            }
            case kProgResync: {
                const long long fresh = fresh_energy_fx<NWP>(sm, th);
                if (tid == 0) sm.st.E_fx = fresh;
                break;
            }
            case kProgPass: {
                if (tid == 0 && args.a_in) sm.st.a = args.a_in[lat];
                __syncthreads();
                if (args.pass_kind == 2)   // multicanonical heat-bath pass at slope a0
                    run_pass<NWP, FAST>(sm, th, 2, (float)args.muca_a0, kTagSweep, 1,
                                        args.class_mask, &args);
                else if (args.pass_kind == 3)   // the end of a composite sweep
                    end_of_sweep<NWP>(sm, th, false);
                else
                    run_pass<NWP, FAST>(sm, th, args.pass_kind, (float)sm.st.a, kTagSweep,
                                        args.block, args.class_mask);
                break;
            }
            case kProgMuca: {
                // one multicanonical composite sweep (Sec. 2.6): heat-bath pass
                // for the weight 1/rho~, n_or overrelaxation passes (they keep
                // E, so every weight of E takes them), resync, energy history
                run_pass<NWP, FAST>(sm, th, 2, (float)args.muca_a0, kTagSweep, 1, 0xFF, &args);
                for (int k = 0; k < args.n_or; ++k)
                    run_pass<NWP, FAST>(sm, th, 1, 0.0f, kTagSweep, 1, 0xFF, nullptr, false);
                end_of_sweep<NWP>(sm, th, false);
                if (tid == 0 && args.e_hist)
                    args.e_hist[(size_t)j * (size_t)args.n_lat + (size_t)lat] =
                        (double)sm.st.E_fx * kInvFx;
                break;
            }
            case kProgBegin: {
                if (tid == 0) {
                    if (args.a_in) sm.st.a = args.a_in[lat];
                    sm.st.sum_dE = 0.0;
                    sm.st.sum_dE2 = 0.0;
                    sm.st.n_meas = 0;
                }
                break;
            }
            case kProgFinish:
                end_of_sweep<NWP>(sm, th, args.measure != 0);
                break;
            case kProgUpdate:
                if (tid == 0) rm_update(sm.st, args, lat);
                break;
            default:
                break;
        }
        __syncthreads();
        if (tid == 0) {
            sm.st.caps += sm.cap_cnt;
            args.lats[lat] = sm.st;
            __threadfence();
            st_release(done + slot, (unsigned)(j + 1));
        }
        __syncthreads();
    }
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

// Dynamic shared memory of one kernel variant: the two stage column sets.
template <int NWP>
constexpr size_t stage_bytes() { return 2u * kStaged * (NWP + 1) * 32 * sizeof(float); }

// Resident CTAs of one kernel variant under a shared-memory carve-out
// preference (carveout: percent of the unified L1/shared storage, or -1 for
// the driver's default).  Queried once per process, device and carve-out; the
// query also sets the variant's dynamic shared memory limit and carve-out (a
// property of the kernel function in this process, so the last configured
// carve-out of a variant applies to every handle that launches it).
template <int NWP, bool FAST>
int resident_ctas(int carveout)
{
    static int cached[64][4] = {};
    static int applied[64] = {};   // carve-out index + 1 last applied per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const int ci = carveout < 0 ? 0 : carveout <= 50 ? 1 : carveout <= 75 ? 2 : 3;
    if (applied[dev] != ci + 1) {
        cudaFuncSetAttribute(llr_kernel<NWP, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)stage_bytes<NWP>());
        const int pct = ci == 0 ? (int)cudaSharedmemCarveoutDefault : ci == 1 ? 50 : ci == 2 ? 75 : 100;
        cudaFuncSetAttribute(llr_kernel<NWP, FAST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             pct);
        applied[dev] = ci + 1;
    }
    if (cached[dev][ci] == 0) {
        int per_sm = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, llr_kernel<NWP, FAST>,
                                                      (NWP + 1) * 32, stage_bytes<NWP>());
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev][ci] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    return cached[dev][ci];
}

template <int NWP, bool FAST>
cudaError_t launch_t(const KernelArgs &a, int carveout, cudaStream_t s, int *grid_out)
{
    const bool multi = a.program == kProgSweeps || a.program == kProgRM || a.program == kProgMuca;
    const long long items = (long long)a.n_lat * (multi ? (a.n_therm + a.n_meas) : 1);
    if (items <= 0) return cudaSuccess;
    const long long cap = resident_ctas<NWP, FAST>(carveout);
    const int grid = (int)(items < cap ? items : cap);
    if (grid_out) *grid_out = grid;
    // the item counter and the done counters; the error word sync[0] is left
    // alone (sticky until the host reads and clears it)
    cudaError_t e = cudaMemsetAsync(a.sync + 1, 0, sizeof(unsigned) * (size_t)(1 + a.n_lat), s);
    if (e != cudaSuccess) return e;
    llr_kernel<NWP, FAST><<<grid, (NWP + 1) * 32, stage_bytes<NWP>(), s>>>(a);
    return cudaGetLastError();
}

}  // namespace

void prime_launch(const LaunchCfg &cfg)
{
    const bool f = cfg.fast_math != 0;
    const int c = cfg.carveout;
    switch (cfg.threads) {
        case 128: f ? resident_ctas<3, true>(c) : resident_ctas<3, false>(c); break;
        case 160: f ? resident_ctas<4, true>(c) : resident_ctas<4, false>(c); break;
        case 192: f ? resident_ctas<5, true>(c) : resident_ctas<5, false>(c); break;
        case 512: f ? resident_ctas<15, true>(c) : resident_ctas<15, false>(c); break;
        default: f ? resident_ctas<7, true>(c) : resident_ctas<7, false>(c); break;
    }
}

cudaError_t launch_llr(const KernelArgs &args, const LaunchCfg &cfg, cudaStream_t s, int *grid_out)
{
    if (args.n_lat <= 0) return cudaSuccess;
    KernelArgs a = args;
    a.ring = cfg.ring;
    const bool f = cfg.fast_math != 0;
    const int c = cfg.carveout;
    switch (cfg.threads) {
        case 128: return f ? launch_t<3, true>(a, c, s, grid_out) : launch_t<3, false>(a, c, s, grid_out);
        case 160: return f ? launch_t<4, true>(a, c, s, grid_out) : launch_t<4, false>(a, c, s, grid_out);
        case 192: return f ? launch_t<5, true>(a, c, s, grid_out) : launch_t<5, false>(a, c, s, grid_out);
        case 512: return f ? launch_t<15, true>(a, c, s, grid_out) : launch_t<15, false>(a, c, s, grid_out);
        default: return f ? launch_t<7, true>(a, c, s, grid_out) : launch_t<7, false>(a, c, s, grid_out);
    }
}

__global__ void step_increment_kernel(int *step)
{
    *step += 1;
}

cudaError_t launch_step_increment(int *step, cudaStream_t s)
{
    step_increment_kernel<<<1, 1, 0, s>>>(step);
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
