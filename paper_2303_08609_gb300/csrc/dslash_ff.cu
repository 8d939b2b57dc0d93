// Float-float hopping kernel: Eq. 1 with every real carried as hi + lo of two
// floats (about 48 significant bits from FP32 operations), spinors in SpFF and
// links in LkFF18. FP64-class accuracy without the FP64 pipe.
//
// Float-float arithmetic costs ~10-15 FP32 instructions per operation, so a
// fully unrolled site (eight directions, each with its own projector) is
// ~12k instructions, far more than the SM's instruction caches hold: profiled,
// warps spent most cycles waiting for instructions. Here the eight directions
// run through ONE loop body: the direction's projector and reconstruction are
// selected at run time from a unit factor (+-1 or +-i) and a spin index (exact
// operations in float-float), and the backward hop conjugate-transposes its
// link in registers, so one copy of the matrix-vector code serves all eight.
#include "weo_internal.h"

namespace weo {

// a + b without the final renormalisation: the sum of the high parts is
// error-free and its error joins the low parts. hi + lo keeps the value to
// ~2^-44 relative to the operands even when lo is no longer below half an ulp
// of hi, which the next operations accept; the accumulators are renormalised
// once at the end.
__device__ __forceinline__ ff ff_add_nr(ff a, ff b)
{
    float s, e;
    ff_two_sum(a.hi, b.hi, s, e);
    return ff(s, __fadd_rn(__fadd_rn(a.lo, b.lo), e));
}
__device__ __forceinline__ cx<ff> cadd_nr(cx<ff> a, cx<ff> b) { return {ff_add_nr(a.r, b.r), ff_add_nr(a.i, b.i)}; }

// sum of the exact products (p_k, e_k) as in the twice-working-precision dot
// product of Ogita, Rump and Oishi (2005): the p_k are added with error-free
// two-sums, every rounding error and every e_k is collected in FP32, and the
// result is renormalised once
template <int N>
__device__ __forceinline__ ff ff_sum_products(const ff (&t)[N])
{
    float s = t[0].hi, err = t[0].lo;
#pragma unroll
    for (int k = 1; k < N; ++k) {
        float e;
        ff_two_sum(s, t[k].hi, s, e);
        err = __fadd_rn(err, __fadd_rn(e, t[k].lo));
    }
    float hi, lo;
    ff_two_sum(s, err, hi, lo);  // s may have cancelled below err
    return ff(hi, lo);
}

// z * c for a unit c: rot selects c = +-i (else +-1), neg the sign
__device__ __forceinline__ cx<ff> unit_mul(cx<ff> z, bool rot, bool neg)
{
    cx<ff> r = rot ? cx<ff>{-z.i, z.r} : z;
    return neg ? cx<ff>{-r.r, -r.i} : r;
}

// Projector (1 - S gamma_mu) and reconstruction in the chiral basis, as unit
// factors: h_0 = psi_0 + c0 psi_j0, h_1 = psi_1 + c1 psi_j1 ;
// out_2 += d2 chi_k2, out_3 += d3 chi_k3 (out_0 += chi_0, out_1 += chi_1).
struct DirCoef {
    bool rot0, neg0, rot1, neg1;  // c0, c1
    int j0, j1;
    bool rot2, neg2, rot3, neg3;  // d2, d3
    int k2, k3;
};

__device__ __forceinline__ DirCoef dir_coef(int mu, int S)
{
    const bool sp = S > 0;
    DirCoef c;
    switch (mu) {
    case 0:  // A = -i sigma_1
        c = {true, !sp, true, !sp, 3, 2, true, sp, true, sp, 1, 0};
        break;
    case 1:  // A = -i sigma_2
        c = {false, !sp, false, sp, 3, 2, false, sp, false, !sp, 1, 0};
        break;
    case 2:  // A = -i sigma_3
        c = {true, !sp, true, sp, 2, 3, true, sp, true, !sp, 0, 1};
        break;
    default:  // A = 1
        c = {false, sp, false, sp, 2, 3, false, sp, false, sp, 0, 1};
        break;
    }
    return c;
}

template <bool Dag, bool Axpy>
__device__ __forceinline__ void hop_site_ff(const HopParams &p, const int i, const int rhs)
{
    constexpr int S0 = Dag ? -1 : 1;
    int rem = i;
    const int xh = rem % p.lxh;
    rem /= p.lxh;
    const int y = rem % p.ly;
    rem /= p.ly;
    const int z = rem % p.lz;
    const int t = rem / p.lz;
    const int par = (y + z + t + p.out_parity) & 1;
    const int op = p.out_parity, in_par = op ^ 1;
    const int sy = p.lxh, sz = p.lxh * p.ly, st = p.lxh * p.ly * p.lz;
    const int row = i - xh;
    const int xp = par ? (xh + 1 == p.lxh ? 0 : xh + 1) : xh;
    const int xm = par ? xh : (xh == 0 ? p.lxh - 1 : xh - 1);
    const int n_xp = row + xp, n_xm = row + xm;
    const int n_yp = i + (y + 1 == p.ly ? -(p.ly - 1) * sy : sy);
    const int n_ym = i + (y == 0 ? (p.ly - 1) * sy : -sy);
    const int n_zp = i + (z + 1 == p.lz ? -(p.lz - 1) * sz : sz);
    const int n_zm = i + (z == 0 ? (p.lz - 1) * sz : -sz);
    const int n_tp = i + (t + 1 == p.lt ? -(p.lt - 1) * st : st);
    const int n_tm = i + (t == 0 ? (p.lt - 1) * st : -st);
    const char *in = static_cast<const char *>(p.in) + rhs * p.in_stride;

    cx<ff> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {ff(0), ff(0)};

#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int nb = d == 0 ? n_xp : d == 1 ? n_xm : d == 2 ? n_yp : d == 3 ? n_ym
                     : d == 4 ? n_zp : d == 5 ? n_zm : d == 6 ? n_tp : n_tm;
        // forward: U_mu(x) at this site; backward: U_mu(x - mu)^dag at the neighbour
        cx<ff> U[3][3];
        LkFF18::load(p.gauge + (2 * mu + (fwd ? op : in_par)) * p.gauge_pb, p.vh, fwd ? i : nb, U);
        if (!fwd) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = a; b < 3; ++b) {
                    const cx<ff> u = U[a][b], v = U[b][a];
                    U[a][b] = {v.r, -v.i};
                    U[b][a] = {u.r, -u.i};
                }
        }
        cx<ff> v[12];
        SpFF::load(in, p.vh, nb, v);
        const DirCoef c = dir_coef(mu, fwd ? S0 : -S0);
        // h[s][colour] = psi_s + c_s psi_{j_s}; spin-colour index k = 3 spin + colour
        cx<ff> h[2][3];
#pragma unroll
        for (int col = 0; col < 3; ++col) {
            const cx<ff> a0 = unit_mul(c.j0 == 2 ? v[6 + col] : v[9 + col], c.rot0, c.neg0);
            const cx<ff> a1 = unit_mul(c.j1 == 2 ? v[6 + col] : v[9 + col], c.rot1, c.neg1);
            h[0][col] = cadd_nr(v[col], a0);
            h[1][col] = cadd_nr(v[3 + col], a1);
        }
        // w = U h: six exact real products per component, summed pairwise
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            cx<ff> w[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ff re[6], im[6];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    re[2 * b] = ff_prod(U[a][b].r, h[s][b].r);
                    re[2 * b + 1] = ff_prod(-U[a][b].i, h[s][b].i);
                    im[2 * b] = ff_prod(U[a][b].r, h[s][b].i);
                    im[2 * b + 1] = ff_prod(U[a][b].i, h[s][b].r);
                }
                w[a] = {ff_sum_products(re), ff_sum_products(im)};
            }
            // out_s += w ; out_{2,3} += d w for the spin row whose k equals s
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                acc[3 * s + a] = cadd_nr(acc[3 * s + a], w[a]);
                if (c.k2 == s) acc[6 + a] = cadd_nr(acc[6 + a], unit_mul(w[a], c.rot2, c.neg2));
                if (c.k3 == s) acc[9 + a] = cadd_nr(acc[9 + a], unit_mul(w[a], c.rot3, c.neg3));
            }
        }
    }

#pragma unroll
    for (int k = 0; k < 12; ++k) {  // renormalise the accumulators (hi may have cancelled)
        float hi, lo;
        ff_two_sum(acc[k].r.hi, acc[k].r.lo, hi, lo);
        acc[k].r = ff(hi, lo);
        ff_two_sum(acc[k].i.hi, acc[k].i.lo, hi, lo);
        acc[k].i = ff(hi, lo);
    }
    if (Axpy) {
        cx<ff> xv[12];
        SpFF::load(static_cast<const char *>(p.x) + rhs * p.x_stride, p.vh, i, xv);
        const ff a(p.a);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            acc[k].r = fma(a, acc[k].r, xv[k].r);
            acc[k].i = fma(a, acc[k].i, xv[k].i);
        }
    }
    SpFF::store(static_cast<char *>(p.out) + rhs * p.out_stride, p.vh, i, acc);
}

// three CTAs of 128 threads per SM (168 registers, no spills): measured
// 2.17 TFlop/s at 32^3 x 64 against 1.97 / 2.11 / 1.81 for two, four or five
template <bool Dag, bool Axpy>
__global__ void __launch_bounds__(128, 3) hop_kernel_ff(const HopParams p)
{
    const int b = p.reverse ? (int)gridDim.x - 1 - (int)blockIdx.x : (int)blockIdx.x;
    const int i = b * blockDim.x + threadIdx.x;
    if (i >= p.vh) return;
    hop_site_ff<Dag, Axpy>(p, i, blockIdx.y);
}

template <bool Dag, bool Axpy>
static int launch_ff(const HopParams &p, cudaStream_t s)
{
    dim3 grid((unsigned)((p.vh + 127) / 128), (unsigned)p.nrhs);
    hop_kernel_ff<Dag, Axpy><<<grid, 128, 0, s>>>(p);
    WEO_CUDA(cudaGetLastError());
    return WEO_OK;
}

int launch_hop_ff(bool dag, bool axpy, const HopParams &p, const LaunchCfg &, cudaStream_t s)
{
    if (dag) return axpy ? launch_ff<true, true>(p, s) : launch_ff<true, false>(p, s);
    return axpy ? launch_ff<false, true>(p, s) : launch_ff<false, false>(p, s);
}

}  // namespace weo
