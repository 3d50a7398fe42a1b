// Non-local Kleinman-Bylander pseudopotential matrix V^NL (Eqs. 2.3-2.4,
// Supp. A.2.2).  The KB operator of atom C is separable,
// v_nl^C(r, r') = sum_p e_p chi_p(r) chi_p(r'), so the paper's two grid stages
// (psi_Cb = v_nl^C phi_b h^3 on the atom's window, then V^C_ab = phi_a .
// psi_Cb h^3) reduce to the grid projections
//   B_pb = h^3 sum_{g in W_p and W_b} chi_p(r_g) phi_b(r_g),
//   V^NL = B^T diag(e) B.
// Projectors are Cartesian Gaussians like the basis functions, with cubic
// windows from the same rule (Eq. A.4), so both factors are products of
// one-dimensional tables and every projection is a product of three
// one-dimensional sums over the intersection of the two windows: the same
// grid sum as over the 3D box, at O(W) cost per pair.  V^NL is formed once
// per geometry (the paper: "only once in the beginning").
#include "dft_internal.cuh"

namespace dft {
namespace {

// one thread per (projector p, basis function b): B[p][b] and E B[p][b]
__global__ void __launch_bounds__(256) k_nl_project(const Fn* __restrict__ fn, const double* __restrict__ tab, int W,
                                                    const Fn* __restrict__ pj, const double* __restrict__ ptab,
                                                    int Wp, const double* __restrict__ e, int K, int np, double h3,
                                                    double* __restrict__ B, double* __restrict__ EB) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)np * K) return;
    const int p = (int)(idx / K), b = (int)(idx % K);
    const Fn P = pj[p], F = fn[b];
    double prod = h3;
    for (int d = 0; d < 3 && prod != 0.0; ++d) {
        const int lo = max(P.lo[d], F.lo[d]), hi = min(P.hi[d], F.hi[d]);
        double s = 0.0;
        const double* tp = ptab + ((long long)p * 3 + d) * Wp - P.lo[d];
        const double* tb = tab + ((long long)b * 3 + d) * W - F.lo[d];
        for (int i = lo; i <= hi; ++i) s = fma(tp[i], tb[i], s);
        prod *= s;
    }
    B[idx] = prod;
    EB[idx] = e[p] * prod;
}

}  // namespace

void launch_nonlocal(const Ctx& c, cudaStream_t s) {
    const int np = (int)c.pj_host.size();
    // the projectors' one-dimensional tables (same kernel as the basis tables)
    launch_build_tables_for(c, c.d_pj, np, c.pj_w, c.d_pjtab, s);
    const long long n = (long long)np * c.Kt;
    k_nl_project<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(c.d_fn, c.d_tab, c.tab_w, c.d_pj, c.d_pjtab, c.pj_w,
                                                            c.d_pje, c.Kt, np, c.h * c.h * c.h, c.d_nlB, c.d_nlEB);
    check_launch("nl_project");
    // V^NL = B^T (E B) from the np x K_t projections of the basis terms,
    // contracted to the functions where they are sums of terms
    double* out = c.contracted ? c.d_Mt : c.d_VNL;
    dgemm('T', 'N', c.Kt, c.Kt, np, 1.0, c.d_nlB, c.Kt, c.d_nlEB, c.Kt, 0.0, out, c.Kt, s);
    if (c.contracted) launch_contract(c, c.d_Mt, c.d_VNL, s);
}

}  // namespace dft
