// tmm_field.cu -- field intensity profile inside every layer.
//
// |E(z) / E_inc|^2 at the depths z_k = (k + 1/2) d_j / n_z of every layer j,
// from the right-to-left sweep of the forward kernel (Eqs. 1-4).  In layer j
// the field is a forward wave a(z) = a_L e^{i kappa z} and a backward wave
// b(z) = b_R e^{i kappa (d - z)} (kappa = 2 pi q_j / lambda), each written
// from the boundary it decays away from: a_L is the sweep's forward amplitude
// at the left boundary (after the layer's phase), b_R its backward amplitude
// at the right boundary (before the phase).  Both are scaled amplitudes; the
// scalars dropped by the sweep are complex but common to the pair at each
// step, so with the incident amplitude set to 1 only their moduli enter:
//   |rho|^2 = 2^{LY - LY_0} (D_0 / D) / |x_0[0]|^2
// (D = prod 4 |k_i|^2 with the power-of-two rescalings, LY = sum of
// 2 Im(delta_i) log2(e) over the layers passed, both at the point where the
// amplitude was taken).  s: |E|^2 = |a + b|^2; p (H_y amplitudes):
// |E|^2 = (|q|^2 |a - b|^2 + beta^2 |a + b|^2) / |n|^4, times n_0^2 for the
// incident E = H / n_0.
#include <cuda_runtime.h>

#include <algorithm>

#include "tmm_device.cuh"
#include "tmm_internal.h"

namespace tmm {

namespace {

constexpr int kFieldThreads = 256;
constexpr int kFieldMaxLayers = 127;

// One polarisation's amplitudes of layer j with their scale bookkeeping.
template <typename R> struct Amp {
    Cx<R> aL, bR;  // forward at the left boundary, backward at the right boundary
    R mL, mR;      // mantissas of D where each was taken
    int eL, eR;    // exponents of D
    R lyL, lyR;    // LY where each was taken
};

template <typename R> __device__ __forceinline__ void dmul_f(R &m, int &e, R v)
{
    m *= v;
    renorm_scalar(m, e);
}

template <typename R, int POL, int KMAX>
__global__ void __launch_bounds__(kFieldThreads) tmm_field_kernel(const tmm_problem p, int n_z, int TL, int TT,
                                                                  int n_lt, int n_tt, R *__restrict__ Eout)
{
    extern __shared__ __align__(16) unsigned char smem[];
    StageA<R> *sa = reinterpret_cast<StageA<R> *>(smem);
    StageB<R> *sb = reinterpret_cast<StageB<R> *>(sa + (size_t)(p.L_max + 2) * TL);
    R *n0s = reinterpret_cast<R *>(sb + (size_t)(p.L_max + 2) * TL);

    const long long item = blockIdx.x;
    const int per_stack = n_lt * n_tt;
    const int s = (int)(item / per_stack);
    const int rr = (int)(item - (long long)s * per_stack);
    const int lt = rr / n_tt, ttile = rr % n_tt;
    const int tid = threadIdx.y * TL + threadIdx.x, nthr = TL * TT;
    const int L = layers_of(p, s);
    const int l0 = lt * TL;
    if (L >= 0) fill_stage<R>(p, s, L, l0, TL, sa, sb, n0s, tid, nthr);
    __syncthreads();
    const int tl = threadIdx.x, l = l0 + tl, a_ = ttile * TT + threadIdx.y;
    if (l >= p.n_lambda || a_ >= p.n_theta) return;  // no barrier follows

    const long long tplane = (long long)p.n_theta * p.n_lambda;
    const long long pt = (long long)a_ * p.n_lambda + l;
    const long long zplane = (long long)n_z * tplane;             // one layer
    const long long splane = (long long)p.L_max * zplane;          // one stack
    const long long Ppol = (long long)p.S * splane;
    const int nplanes = (POL & 4) ? 1 : ((POL & 1) + ((POL >> 1) & 1));
    auto store = [&](int pi, int j, int kz, R v) {
        Eout[pi * Ppol + (long long)s * splane + (long long)j * zplane + (long long)kz * tplane + pt] = v;
    };

    const R n0 = L >= 0 ? n0s[tl] : nan_w<R>();
    R sth, cth;
    sincos_w(((const R *)p.theta)[a_], &sth, &cth);
    const R beta = n0 * sth, c0 = n0 * cth, q0sq = c0 * c0;
    const bool grazing = beta >= n0;
    if (L < 0 || !(n0 == n0) || grazing) {
        // exact grazing: no field enters the stack
        const R fill = grazing ? R(0) : nan_w<R>();
        for (int pi = 0; pi < nplanes; ++pi)
            for (int j = 0; j < p.L_max; ++j)
                for (int kz = 0; kz < n_z; ++kz) store(pi, j, kz, (j < L || L < 0) ? fill : R(0));
        return;
    }
    constexpr int RN = RenormEvery<R>::value;
    const R yi_max = R(kImDeltaMax / kTwoPi);
    const R kLY = R(2.0 * kTwoPi * kLog2e);
    Amp<R> as[(POL & 1) ? KMAX : 1], ap[(POL & 2) ? KMAX : 1];
    StageA<R> A = sa[(L + 1) * TL + tl];
    R absz;
    Cx<R> q_nx = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
    Cx<R> g_nx = cmul(q_nx, Cx<R>{A.in2x, A.in2y});
    Cx<R> s0 = {R(1), R(0)}, s1 = {R(0), R(0)}, p0 = s0, p1 = s1;
    R Dsm = R(1), Dpm = R(1), LY = R(0);
    int Dse = 0, Dpe = 0, cnt = 0;
    for (int j = L; j >= 1; --j) {
        A = sa[j * TL + tl];
        const StageB<R> B = sb[j * TL + tl];
        const Cx<R> q = forward_root(Cx<R>{A.d2x + q0sq, A.n2y}, &absz);
        const R yr = B.dl * q.x;
        const R yi = fmin(B.dl * q.y, yi_max);
        R sn, cs;
        sincos_turn(yr - rint_w(yr), &sn, &cs);
        const R E2 = exp_m2_turn(yi);
        const Cx<R> emi = {cs, -sn}, epi = {E2 * cs, E2 * sn};
        const Cx<R> g = cmul(q, Cx<R>{A.in2x, A.in2y});
        if (POL & 1) {
            interface_pair(q, q_nx, s0, s1);
            dmul_f(Dsm, Dse, R(4) * absz);
            as[j].bR = s1, as[j].mR = Dsm, as[j].eR = Dse, as[j].lyR = LY;
            s0 = cmul(emi, s0);
            s1 = cmul(epi, s1);
        }
        if (POL & 2) {
            interface_pair(g, g_nx, p0, p1);
            dmul_f(Dpm, Dpe, R(4) * absz * B.ain2);
            ap[j].bR = p1, ap[j].mR = Dpm, ap[j].eR = Dpe, ap[j].lyR = LY;
            p0 = cmul(emi, p0);
            p1 = cmul(epi, p1);
        }
        LY += kLY * yi;
        if (++cnt == RN) {
            cnt = 0;
            if (POL & 1) {
                int k = 0;
                renorm_pair(s0, s1, k);
                Dse -= 2 * k;
            }
            if (POL & 2) {
                int k = 0;
                renorm_pair(p0, p1, k);
                Dpe -= 2 * k;
            }
        }
        if (POL & 1) as[j].aL = s0, as[j].mL = Dsm, as[j].eL = Dse, as[j].lyL = LY;
        if (POL & 2) ap[j].aL = p0, ap[j].mL = Dpm, ap[j].eL = Dpe, ap[j].lyL = LY;
        q_nx = q;
        g_nx = g;
    }
    // interface 0 | 1: the incident amplitude x_0[0]
    A = sa[tl];
    const Cx<R> q0 = {c0, R(0)};
    const Cx<R> g0 = cmul(q0, Cx<R>{A.in2x, A.in2y});
    R pre[2] = {R(0), R(0)};
    int e0[2] = {0, 0};
    if (POL & 1) {
        interface_pair(q0, q_nx, s0, s1);
        dmul_f(Dsm, Dse, R(4) * c0 * c0);
        pre[0] = Dsm / abs2(s0);
        e0[0] = Dse;
    }
    if (POL & 2) {
        interface_pair(g0, g_nx, p0, p1);
        dmul_f(Dpm, Dpe, R(4) * abs2(g0));
        pre[1] = Dpm / abs2(p0) * n0 * n0;  // the incident E = H / n_0
        e0[1] = Dpe;
    }
    // |rho| of an amplitude taken at (m, e, ly)
    auto rho = [&](int k, R m, int e, R ly) {
        const R w = ly - LY;  // <= 0
        const R wn = floor_w(w);
        return sqrt(ldexp_w(pre[k] / m * exp2_w(w - wn), e0[k] - e + (int)wn));
    };
    for (int j = 1; j <= L; ++j) {
        const StageA<R> Aj = sa[j * TL + tl];
        const StageB<R> Bj = sb[j * TL + tl];
        const Cx<R> q = forward_root(Cx<R>{Aj.d2x + q0sq, Aj.n2y}, &absz);
        const R n4 = R(1) / Bj.ain2;  // |n_j|^4
        Cx<R> fa[2], fb[2];
        if (POL & 1) {
            fa[0] = scale(rho(0, as[j].mL, as[j].eL, as[j].lyL), as[j].aL);
            fb[0] = scale(rho(0, as[j].mR, as[j].eR, as[j].lyR), as[j].bR);
        }
        if (POL & 2) {
            fa[1] = scale(rho(1, ap[j].mL, ap[j].eL, ap[j].lyL), ap[j].aL);
            fb[1] = scale(rho(1, ap[j].mR, ap[j].eR, ap[j].lyR), ap[j].bR);
        }
        for (int kz = 0; kz < n_z; ++kz) {
            const R f = (R(kz) + R(0.5)) / R(n_z);  // z / d
            // e^{i kappa z} and e^{i kappa (d - z)} in turns of the layer phase
            R s1n, c1s, s2n, c2s;
            const R y1r = Bj.dl * q.x * f, y2r = Bj.dl * q.x * (R(1) - f);
            sincos_turn(y1r - rint_w(y1r), &s1n, &c1s);
            sincos_turn(y2r - rint_w(y2r), &s2n, &c2s);
            const R m1 = sqrt(exp_m2_turn(Bj.dl * q.y * f)), m2 = sqrt(exp_m2_turn(Bj.dl * q.y * (R(1) - f)));
            const Cx<R> ez = {m1 * c1s, m1 * s1n}, edz = {m2 * c2s, m2 * s2n};
            R v[2] = {R(0), R(0)};
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(POL & (1 << k))) continue;
                const Cx<R> af = cmul(fa[k], ez), bf = cmul(fb[k], edz);
                v[k] = k == 0 ? abs2(af + bf) : (abs2(q) * abs2(af - bf) + beta * beta * abs2(af + bf)) / n4;
            }
            if (POL & 4) {
                store(0, j - 1, kz, R(0.5) * (v[0] + v[1]));
            } else {
                int pi = 0;
                if (POL & 1) store(pi++, j - 1, kz, v[0]);
                if (POL & 2) store(pi, j - 1, kz, v[1]);
            }
        }
    }
    for (int pi = 0; pi < nplanes; ++pi)
        for (int j = L; j < p.L_max; ++j)
            for (int kz = 0; kz < n_z; ++kz) store(pi, j, kz, R(0));
}

size_t field_smem(const tmm_problem *p, int TL)
{
    const size_t r = real_size(p->prec);
    return (size_t)(p->L_max + 2) * TL * (6 * r) + (size_t)TL * r;
}

template <typename R, int POL, int KMAX>
tmm_status launch_field_k(const tmm_problem *p, int n_z, int TL, int TT, int n_lt, int n_tt, long long items,
                          size_t smem, R *E, cudaStream_t st)
{
    auto k = tmm_field_kernel<R, POL, KMAX>;
    if (smem > 48 * 1024) {
        static int set_bytes[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e);
        if (dev < 0 || dev >= 64) return TMM_ERR_UNSUPPORTED;
        if (set_bytes[dev] < (int)smem) {
            e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e);
            set_bytes[dev] = (int)smem;
        }
    }
    k<<<(unsigned)items, dim3(TL, TT), smem, st>>>(*p, n_z, TL, TT, n_lt, n_tt, E);
    return check_launch();
}

template <typename R, int POL>
tmm_status launch_field_km(const tmm_problem *p, int n_z, int TL, int TT, int n_lt, int n_tt, long long items,
                           size_t smem, R *E, cudaStream_t st)
{
    const int need = p->L_max + 2;
    if (need <= 18) return launch_field_k<R, POL, 18>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    if (need <= 34) return launch_field_k<R, POL, 34>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    if (need <= 66) return launch_field_k<R, POL, 66>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    return launch_field_k<R, POL, kFieldMaxLayers + 2>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
}

template <typename R>
tmm_status launch_field_prec(const tmm_problem *p, int n_z, int TL, int TT, int n_lt, int n_tt, long long items,
                             size_t smem, void *E_, cudaStream_t st)
{
    R *E = static_cast<R *>(E_);
    switch (p->pol_mask) {
    case 1: return launch_field_km<R, 1>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    case 2: return launch_field_km<R, 2>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    case 3: return launch_field_km<R, 3>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    case 7: return launch_field_km<R, 7>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
    default: return TMM_ERR_INVALID_ARG;
    }
}

}  // namespace

}  // namespace tmm

using namespace tmm;

extern "C" TMM_API tmm_status tmm_field_profile(const tmm_problem *p, int32_t n_z, void *E, void *stream)
{
    tmm_status s = validate_problem(p);
    if (s != TMM_OK) return s;
    if (p->prec == TMM_F64X) return TMM_ERR_UNSUPPORTED;
    if (p->L_max > kFieldMaxLayers) return TMM_ERR_UNSUPPORTED;
    if (n_z < 1) return TMM_ERR_INVALID_ARG;
    const long long pts = (long long)p->S * p->n_lambda * p->n_theta;
    if (pts == 0 || p->L_max == 0) return TMM_OK;
    if (!E) return TMM_ERR_INVALID_ARG;
    DeviceInfo di;
    s = device_info(&di);
    if (s != TMM_OK) return s;
    const int TT = std::min(p->n_theta, 32);
    int TL = 1;
    while (TL * TT * 2 <= kFieldThreads) TL *= 2;
    while (TL > 1 && TL / 2 >= p->n_lambda) TL /= 2;
    while (TL > 1 && field_smem(p, TL) > (size_t)di.max_smem_optin) TL /= 2;
    const size_t smem = field_smem(p, TL);
    if (smem > (size_t)di.max_smem_optin) return TMM_ERR_UNSUPPORTED;
    const int n_lt = (p->n_lambda + TL - 1) / TL, n_tt = (p->n_theta + TT - 1) / TT;
    const long long items = (long long)p->S * n_lt * n_tt;
    if (items > 0x7fffffffLL) return TMM_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return p->prec == TMM_F64 ? launch_field_prec<double>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st)
                              : launch_field_prec<float>(p, n_z, TL, TT, n_lt, n_tt, items, smem, E, st);
}
