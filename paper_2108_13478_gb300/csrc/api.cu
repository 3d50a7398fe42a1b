// C ABI of libdft (include/dft.h): context set-up, workspace layout and the
// host-side orchestration of the SCF cycle (Supp. A.3).  Every numerical
// step runs in the kernels of k_*.cu; the host only sizes the problem, picks
// the Chebyshev order and enqueues work.
#include "dft_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <new>
#include <thread>

using namespace dft;

std::atomic<unsigned long long> dft::g_launches{0};

namespace {

const char* kVersion = "libdft 0.2 (sm_103a)";
// reuse of mu between SCF cycles, in units of kT (see dft_scf_step)
constexpr double MU_SETTLED = 0.01, MU_REDO = 0.05;

// Window half-length L solving c(L sqrt(zeta), l) = 1 - eta (Eq. A.4).
// c(d, 0) = erf(d), c(d, 1) = 1 - exp(-d^2),
// c(d, 2) = erf(d) - 2 d exp(-d^2) / sqrt(pi).
double window_halfwidth(double zeta, int l, double eta) {
    double d;
    if (l == 1) {
        d = std::sqrt(-std::log(eta));
    } else {
        // 1 - c(d, l), decreasing in d
        auto tail = [l](double x) {
            return l == 0 ? std::erfc(x) : std::erfc(x) + 2.0 * x * std::exp(-x * x) / std::sqrt(M_PI);
        };
        double lo = 0.0, hi = 40.0;
        for (int it = 0; it < 400; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (tail(mid) > eta) lo = mid; else hi = mid;
        }
        d = 0.5 * (lo + hi);
    }
    return d / std::sqrt(zeta);
}

// Table A.1: the real solid harmonics of degree 2 as weights of the
// Cartesian monomials x^i y^j z^k, in the table's order of m (2, 1, 0, -1, -2);
// s and p have one monomial of weight 1 (p in the Cartesian order x, y, z)
struct Mono {
    int i, j, k;
    double w;
};
std::vector<std::vector<Mono>> shell_components(int l, bool spherical) {
    const double r3 = std::sqrt(3.0);
    if (l == 0) return {{{0, 0, 0, 1.0}}};
    if (l == 1) return {{{1, 0, 0, 1.0}}, {{0, 1, 0, 1.0}}, {{0, 0, 1, 1.0}}};
    if (spherical)
        return {{{2, 0, 0, 0.5 * r3}, {0, 2, 0, -0.5 * r3}}, {{1, 1, 0, r3}},
                {{2, 0, 0, -0.5}, {0, 2, 0, -0.5}, {0, 0, 2, 1.0}}, {{0, 1, 1, r3}}, {{1, 0, 1, r3}}};
    return {{{2, 0, 0, 1.0}}, {{0, 2, 0, 1.0}}, {{0, 0, 2, 1.0}},
            {{1, 1, 0, 1.0}}, {{1, 0, 1, 1.0}}, {{0, 1, 1, 1.0}}};
}

// normalisation of x^l exp(-zeta r^2): (2 zeta / pi)^(3/4) (4 zeta)^(l/2) / sqrt((2l - 1)!!)
double monomial_norm(double zeta, int l) {
    const double dfact = l == 2 ? 3.0 : 1.0;
    return std::pow(2.0 * zeta / M_PI, 0.75) * std::pow(4.0 * zeta, 0.5 * l) / std::sqrt(dfact);
}

struct Layout {
    size_t total = 0;
    size_t off(size_t bytes) {
        size_t o = total;
        total += (bytes + 255) & ~size_t(255);
        return o;
    }
};

void validate(const dft_basis_desc* b, const dft_grid_desc* g, const dft_params* p) {
    if (!b || !g || !p) throw Error(DFT_EINVAL, "null descriptor");
    if (b->n_atoms <= 0 || !b->xyz) throw Error(DFT_EINVAL, "no atoms");
    if (b->n_shells <= 0 || !b->shell_atom || !b->shell_l) throw Error(DFT_EINVAL, "no shells");
    if (!b->shell_nprim && !b->shell_exp) throw Error(DFT_EINVAL, "no shell exponents");
    if (b->shell_nprim && (!b->prim_exp || !b->prim_coef)) throw Error(DFT_EINVAL, "contracted shells need prim_exp and prim_coef");
    long long np = 0;
    for (int s = 0; s < b->n_shells; ++s) {
        if (b->shell_atom[s] < 0 || b->shell_atom[s] >= b->n_atoms) throw Error(DFT_EINVAL, "shell_atom out of range");
        if (b->shell_l[s] < 0 || b->shell_l[s] > 2) throw Error(DFT_EINVAL, "only s, p and d shells are supported");
        if (b->shell_nprim) {
            if (b->shell_nprim[s] < 1 || b->shell_nprim[s] > 32) throw Error(DFT_EINVAL, "shell_nprim must be in [1, 32]");
            for (int q = 0; q < b->shell_nprim[s]; ++q)
                if (!(b->prim_exp[np + q] > 0.0)) throw Error(DFT_EINVAL, "primitive exponent must be positive");
            np += b->shell_nprim[s];
        } else if (!(b->shell_exp[s] > 0.0)) {
            throw Error(DFT_EINVAL, "shell exponent must be positive");
        }
    }
    if (!(g->h > 0.0)) throw Error(DFT_EINVAL, "grid spacing must be positive");
    for (int d = 0; d < 3; ++d)
        if (g->n[d] <= 0 || g->n[d] > 4096) throw Error(DFT_EINVAL, "grid size out of range");
    if (!(p->beta > 0.0)) throw Error(DFT_EINVAL, "beta must be positive");
    if (!(p->eta > 0.0 && p->eta < 1.0)) throw Error(DFT_EINVAL, "eta must be in (0, 1)");
    if (p->precision != DFT_PREC_FP64 && p->precision != DFT_PREC_BF16X3 && p->precision != DFT_PREC_FP16X3)
        throw Error(DFT_EINVAL, "unknown precision");
    if (p->cheb_order <= 0 && !(p->cheb_tail_tol > 0.0)) throw Error(DFT_EINVAL, "cheb_tail_tol must be positive");
    if (p->mixer < DFT_MIX_LINEAR || p->mixer > DFT_MIX_PULAY) throw Error(DFT_EINVAL, "unknown mixer");
    if (p->mix_history < 0 || p->mix_history > 16) throw Error(DFT_EINVAL, "mix_history must be in [0, 16]");
    if (p->nl_channels != 0 && p->nl_channels != 1 && p->nl_channels != 4)
        throw Error(DFT_EINVAL, "nl_channels must be 0, 1 (s) or 4 (s and p)");
    if (p->nl_channels && !(p->nl_zeta > 0.0)) throw Error(DFT_EINVAL, "nl_zeta must be positive");
    if (p->xc != DFT_XC_SLATER && p->xc != DFT_XC_PW92) throw Error(DFT_EINVAL, "unknown xc");
}

// functions, windows, tables and tile lists (host part of the set-up)
void build_basis(Ctx& c, const dft_basis_desc* b, const dft_grid_desc* g, const dft_params* p,
                 std::vector<int>* tile_ptr, std::vector<int>* tile_fn) {
    c.n_atoms = b->n_atoms;
    c.h = g->h;
    for (int d = 0; d < 3; ++d) { c.n[d] = g->n[d]; c.origin[d] = g->origin[d]; }
    c.ng = (long long)c.n[0] * c.n[1] * c.n[2];
    c.p = *p;
    c.xyz_host.assign(b->xyz, b->xyz + 3 * b->n_atoms);
    c.fn_host.clear();
    c.fn_atom_host.clear();
    c.term_ptr_host.assign(1, 0);
    int wmax = 1;
    // Every basis function (Eq. A.1) is a sum of Cartesian Gaussian terms,
    // coefficient d_p w^{ijk} (contraction times Table A.1 weight) times the
    // monomial's normalisation; all terms of a function share its window, set
    // by its most diffuse primitive (Supp. A.1.1).  The grid kernels and the
    // closed-form integrals work on the terms; function-level matrices are
    // contracted from them (with the functions' normalisation N_a, formed on
    // the device from the closed-form overlap).  An uncontracted s/p basis has
    // one term per function with its primitive's normalisation: no
    // contraction step at all.
    bool contracted = false;
    long long poff = 0;
    for (int s = 0; s < b->n_shells; ++s) {
        const int a = b->shell_atom[s], l = b->shell_l[s];
        std::vector<std::pair<double, double>> prims;
        if (b->shell_nprim) {
            for (int q = 0; q < b->shell_nprim[s]; ++q) prims.emplace_back(b->prim_exp[poff + q], b->prim_coef[poff + q]);
            poff += b->shell_nprim[s];
        } else {
            prims.emplace_back(b->shell_exp[s], 1.0);
        }
        if (l == 2 || prims.size() > 1 || prims[0].second != 1.0) contracted = true;
        double zmin = prims[0].first;
        for (auto& pr : prims) zmin = std::min(zmin, pr.first);
        const double L = window_halfwidth(zmin, l, p->eta);
        int lo_w[3], hi_w[3];
        const double cc[3] = {b->xyz[3 * a], b->xyz[3 * a + 1], b->xyz[3 * a + 2]};
        for (int d = 0; d < 3; ++d) {
            long long lo = (long long)std::ceil((cc[d] - L - c.origin[d]) / c.h);
            long long hi = (long long)std::floor((cc[d] + L - c.origin[d]) / c.h);
            lo = std::max<long long>(lo, 0);
            hi = std::min<long long>(hi, c.n[d] - 1);
            lo_w[d] = (int)std::min<long long>(lo, c.n[d]);
            hi_w[d] = (int)std::max<long long>(hi, -1);
            wmax = std::max(wmax, hi_w[d] - lo_w[d] + 1);
        }
        for (const auto& comp : shell_components(l, b->spherical != 0)) {
            for (const auto& pr : prims)
                for (const Mono& m : comp) {
                    Fn f{};
                    f.cx = cc[0]; f.cy = cc[1]; f.cz = cc[2];
                    f.zeta = pr.first;
                    f.norm = pr.second * m.w * monomial_norm(pr.first, l);
                    f.px = m.i; f.py = m.j; f.pz = m.k;
                    for (int d = 0; d < 3; ++d) { f.lo[d] = lo_w[d]; f.hi[d] = hi_w[d]; }
                    c.fn_host.push_back(f);
                }
            c.term_ptr_host.push_back((int)c.fn_host.size());
            c.fn_atom_host.push_back(a);
        }
    }
    c.K = (int)c.term_ptr_host.size() - 1;
    c.Kt = (int)c.fn_host.size();
    c.contracted = contracted;
    c.tab_w = wmax;
    for (int d = 0; d < 3; ++d) c.ntile[d] = (c.n[d] + TILE - 1) / TILE;
    c.n_tiles = (long long)c.ntile[0] * c.ntile[1] * c.ntile[2];
    std::vector<int> cnt(c.n_tiles + 1, 0);
    auto each_tile = [&](const Fn& f, auto&& fun) {
        for (int d = 0; d < 3; ++d)
            if (f.lo[d] > f.hi[d]) return;
        for (int tz = f.lo[2] / TILE; tz <= f.hi[2] / TILE; ++tz)
            for (int ty = f.lo[1] / TILE; ty <= f.hi[1] / TILE; ++ty)
                for (int tx = f.lo[0] / TILE; tx <= f.hi[0] / TILE; ++tx)
                    fun(((long long)tz * c.ntile[1] + ty) * c.ntile[0] + tx);
    };
    for (const Fn& f : c.fn_host) each_tile(f, [&](long long t) { cnt[t + 1]++; });
    for (long long t = 0; t < c.n_tiles; ++t) cnt[t + 1] += cnt[t];
    c.tile_nnz = cnt[c.n_tiles];
    c.tile_max = 0;
    for (long long t = 0; t < c.n_tiles; ++t) c.tile_max = std::max(c.tile_max, cnt[t + 1] - cnt[t]);
    if (tile_ptr) {
        *tile_ptr = cnt;
        tile_fn->assign(c.tile_nnz, 0);
        std::vector<int> pos(cnt.begin(), cnt.end() - 1);
        for (int f = 0; f < c.Kt; ++f) each_tile(c.fn_host[f], [&](long long t) { (*tile_fn)[pos[t]++] = f; });
    }
    // KB projectors (Supp. A.2.2): per atom an s Gaussian (and x, y, z p
    // Gaussians) of exponent nl_zeta, unit continuum norm, cube windows by
    // the basis functions' rule (Eq. A.4)
    c.pj_host.clear();
    c.pje_host.clear();
    c.pj_w = 0;
    if (p->nl_channels > 0) {
        const double z = p->nl_zeta, base = std::pow(2.0 * z / M_PI, 0.75);
        for (int a = 0; a < b->n_atoms; ++a)
            for (int q = 0; q < p->nl_channels; ++q) {
                const int l = q == 0 ? 0 : 1;
                Fn f{};
                f.cx = b->xyz[3 * a]; f.cy = b->xyz[3 * a + 1]; f.cz = b->xyz[3 * a + 2];
                f.zeta = z;
                f.norm = l == 0 ? base : base * 2.0 * std::sqrt(z);
                f.px = q == 1; f.py = q == 2; f.pz = q == 3;
                const double L = window_halfwidth(z, l, p->eta);
                const double cc[3] = {f.cx, f.cy, f.cz};
                for (int d = 0; d < 3; ++d) {
                    long long lo = (long long)std::ceil((cc[d] - L - c.origin[d]) / c.h);
                    long long hi = (long long)std::floor((cc[d] + L - c.origin[d]) / c.h);
                    lo = std::max<long long>(lo, 0);
                    hi = std::min<long long>(hi, c.n[d] - 1);
                    f.lo[d] = (int)std::min<long long>(lo, c.n[d]);
                    f.hi[d] = (int)std::max<long long>(hi, -1);
                    c.pj_w = std::max(c.pj_w, f.hi[d] - f.lo[d] + 1);
                }
                c.pj_host.push_back(f);
                c.pje_host.push_back(l == 0 ? p->nl_e_s : p->nl_e_p);
            }
    }
    for (int d = 0; d < 3; ++d) c.Nfft[d] = fft_size(2 * c.n[d]);
    c.nfft_r = (long long)c.Nfft[0] * c.Nfft[1] * c.Nfft[2];
    c.nfft_c = (long long)(c.Nfft[0] / 2 + 1) * c.Nfft[1] * c.Nfft[2];
    c.cheb_cap = 1 << 16;
    if (c.p.precision != DFT_PREC_FP64) {
        c.Kp = tc_pad(c.K);
        c.n_tc_tiles = (int)((tc_tiles(c.K, 256).size() + tc_tiles(c.K, 128).size()) / 2);
        c.tile_cap = std::max(c.n_tc_tiles, 1 << 17);
    }
    c.part_cap = std::max<long long>({2LL * cheb_step_parts(c.K), 2LL * c.tile_cap, 3LL * 1184, 2048, 592LL * 16}) + 64;
    c.pl_hist = c.p.mixer == DFT_MIX_PULAY ? (c.p.mix_history > 0 ? c.p.mix_history : 8) : 0;
}

// carve the workspace; with base == nullptr only the size is computed
size_t carve(Ctx& c, char* base) {
    Layout L;
    size_t K2 = (size_t)c.K * c.K * sizeof(double);
    size_t G = (size_t)c.ng * sizeof(double);
    long long nkc = (long long)(c.n[0] / 2 + 1) * c.n[1] * c.n[2];
    size_t o_fn = L.off(sizeof(Fn) * c.Kt);
    size_t o_tab = L.off(sizeof(double) * (size_t)c.Kt * 3 * c.tab_w);
    size_t o_ttp = 0, o_tpar = 0, o_cn = 0, o_mt = 0;
    if (c.contracted) {
        o_ttp = L.off(sizeof(int) * ((size_t)c.K + 1));
        o_tpar = L.off(sizeof(int) * (size_t)c.Kt);
        o_cn = L.off(sizeof(double) * (size_t)c.K);
        o_mt = L.off(sizeof(double) * (size_t)c.Kt * c.Kt);
    }
    size_t o_tp = L.off(sizeof(int) * (c.n_tiles + 1));
    size_t o_tf = L.off(sizeof(int) * std::max<long long>(1, c.tile_nnz));
    size_t o_xyz = L.off(sizeof(double) * 3 * c.n_atoms);
    size_t o_S = L.off(K2), o_T = L.off(K2), o_Li = L.off(K2), o_A = L.off(K2), o_H = L.off(K2);
    size_t o_X0 = L.off(K2), o_X1 = L.off(K2), o_rho = L.off(K2), o_B = L.off(K2), o_P = L.off(K2);
    size_t o_F = L.off(K2);
    size_t o_vec = L.off(sizeof(double) * 4 * c.K);
    size_t o_scal = L.off(sizeof(double) * SCAL_COUNT);
    size_t o_coef = L.off(sizeof(double) * (5 * (size_t)c.cheb_cap + 64));
    size_t o_mom = L.off(sizeof(double) * c.cheb_cap);
    size_t o_cos = L.off(sizeof(double) * 16 * (size_t)c.cheb_cap);
    size_t o_wk = L.off(sizeof(double) * 4 * (size_t)c.cheb_cap);
    size_t o_part = L.off(sizeof(double) * c.part_cap);
    size_t o_flags = L.off(sizeof(int) * FLAG_COUNT);
    size_t o_vloc = L.off(G), o_nion = L.off(G), o_vks = L.off(G), o_nout = L.off(G), o_gtmp = L.off(G);
    size_t o_fr = L.off(sizeof(double) * c.nfft_r);
    size_t o_fo = L.off(sizeof(double) * c.nfft_r);
    size_t o_gh = L.off(sizeof(double) * c.nfft_c);
    size_t o_fc = L.off(sizeof(cufftDoubleComplex) * c.nfft_c);
    size_t o_kw = L.off(sizeof(double) * nkc);
    size_t o_kc = L.off(sizeof(cufftDoubleComplex) * nkc);
    size_t o_pl = c.pl_hist > 0 ? L.off(sizeof(double) * 2 * (size_t)c.pl_hist * c.ng) : 0;
    size_t o_wdesc = L.off(sizeof(double) * 32 * (size_t)c.n_atoms);
    size_t o_wcoef = L.off(sizeof(double) * 16 * (size_t)c.n_atoms);
    size_t o_wz = L.off(sizeof(float) * 3 * 128 * (size_t)c.n_atoms);
    size_t o_wdc = L.off(sizeof(double) * 16 * (size_t)c.n_atoms);
    const size_t np = c.pj_host.size();
    size_t o_pj = 0, o_pje = 0, o_pjt = 0, o_nlb = 0, o_nleb = 0, o_vnl = 0;
    if (np > 0) {
        o_pj = L.off(sizeof(Fn) * np);
        o_pje = L.off(sizeof(double) * np);
        o_pjt = L.off(sizeof(double) * np * 3 * (size_t)c.pj_w);
        o_nlb = L.off(sizeof(double) * np * (size_t)c.Kt);
        o_nleb = L.off(sizeof(double) * np * (size_t)c.Kt);
        o_vnl = L.off(K2);
    }
    size_t o_h16[2] = {0, 0}, o_x16[4] = {0, 0, 0, 0}, o_rtc = 0, o_tiles = 0, o_systab = 0, o_maps = 0;
    size_t o_cst = 0, o_skf = 0, o_skb = 0, o_cnt = 0, o_macc = 0, o_li16[2] = {0, 0}, o_lt16[2] = {0, 0};
    if (c.Kp > 0) {
        size_t P16 = (size_t)c.Kp * c.Kp * 2;
        for (auto& o : o_h16) o = L.off(P16);
        for (auto& o : o_x16) o = L.off(P16);
        for (auto& o : o_li16) o = L.off(P16);
        for (auto& o : o_lt16) o = L.off(P16);
        o_rtc = L.off((size_t)c.Kp * c.Kp * sizeof(double));
        o_systab = L.off(sizeof(TcSys) * TC_MAX_SYS);
        o_maps = L.off(sizeof(CUtensorMap) * TC_MAPS_PER_SYS * TC_MAX_SYS);
        o_tiles = L.off(sizeof(TcTile) * (size_t)c.tile_cap);
        o_cst = L.off(sizeof(int) * ((size_t)c.tile_cap + 1));
        o_skf = L.off(sizeof(int) * (size_t)c.tile_cap);
        o_skb = L.off(sizeof(float) * (size_t)TC_SK_MAX_CTAS * 256 * 128);
        o_cnt = L.off(sizeof(int) * 3 * (size_t)c.tile_cap);
        o_macc = L.off(sizeof(long long) * (size_t)c.cheb_cap);
    }
    if (base) {
        c.d_fn = (Fn*)(base + o_fn);
        c.d_tab = (double*)(base + o_tab);
        if (c.contracted) {
            c.d_term_ptr = (int*)(base + o_ttp);
            c.d_term_par = (int*)(base + o_tpar);
            c.d_cnorm = (double*)(base + o_cn);
            c.d_Mt = (double*)(base + o_mt);
        }
        c.d_tile_ptr = (int*)(base + o_tp);
        c.d_tile_fn = (int*)(base + o_tf);
        c.d_xyz = (double*)(base + o_xyz);
        c.d_S = (double*)(base + o_S); c.d_T = (double*)(base + o_T); c.d_Linv = (double*)(base + o_Li);
        c.d_A = (double*)(base + o_A); c.d_H = (double*)(base + o_H);
        c.d_X0 = (double*)(base + o_X0); c.d_X1 = (double*)(base + o_X1); c.d_rho = (double*)(base + o_rho);
        c.d_B = (double*)(base + o_B); c.d_P = (double*)(base + o_P); c.d_F = (double*)(base + o_F);
        c.d_vec = (double*)(base + o_vec);
        c.d_scal = (double*)(base + o_scal);
        c.d_coef = (double*)(base + o_coef);
        c.d_mom = (double*)(base + o_mom);
        c.d_cos = (double*)(base + o_cos);
        c.d_wk = (double*)(base + o_wk);
        c.d_part = (double*)(base + o_part);
        c.d_flags = (int*)(base + o_flags);
        c.d_vloc = (double*)(base + o_vloc); c.d_nion = (double*)(base + o_nion);
        c.d_vks = (double*)(base + o_vks); c.d_nout = (double*)(base + o_nout); c.d_gtmp = (double*)(base + o_gtmp);
        c.d_fft_r = (double*)(base + o_fr);
        c.d_fft_o = (double*)(base + o_fo);
        c.d_ghat = (double*)(base + o_gh);
        c.d_fft_c = (cufftDoubleComplex*)(base + o_fc);
        c.d_kerker = (double*)(base + o_kw);
        c.d_kc = (cufftDoubleComplex*)(base + o_kc);
        if (c.pl_hist > 0) c.d_pulay = (double*)(base + o_pl);
        c.d_wdesc = (double*)(base + o_wdesc);
        c.d_wcoef = (double*)(base + o_wcoef);
        c.d_wz = (float*)(base + o_wz);
        c.d_wdc = (double*)(base + o_wdc);
        if (np > 0) {
            c.d_pj = (Fn*)(base + o_pj);
            c.d_pje = (double*)(base + o_pje);
            c.d_pjtab = (double*)(base + o_pjt);
            c.d_nlB = (double*)(base + o_nlb);
            c.d_nlEB = (double*)(base + o_nleb);
            c.d_VNL = (double*)(base + o_vnl);
        }
        if (c.Kp > 0) {
            for (int q = 0; q < 2; ++q) c.d_h16[q] = base + o_h16[q];
            for (int q = 0; q < 4; ++q) c.d_x16[q] = base + o_x16[q];
            for (int q = 0; q < 2; ++q) {
                c.d_li16[q] = base + o_li16[q];
                c.d_lt16[q] = base + o_lt16[q];
            }
            c.d_rho_tc = (float2*)(base + o_rtc);
            c.d_systab = (TcSys*)(base + o_systab);
            c.d_maps = (CUtensorMap*)(base + o_maps);
            c.d_tiles = (TcTile*)(base + o_tiles);
            c.d_cstart = (int*)(base + o_cst);
            c.d_skflag = (int*)(base + o_skf);
            c.d_skbuf = (float*)(base + o_skb);
            c.d_cnt = (int*)(base + o_cnt);
            c.d_macc = (long long*)(base + o_macc);
        }
    }
    return L.total;
}

template <class F>
dft_status guarded(dft_ctx* ctx, F&& f) {
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    try {
        f();
        if (c) c->err.clear();
        return DFT_OK;
    } catch (const Error& e) {
        if (c) c->err = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        if (c) c->err = "host allocation failed";
        return DFT_ENOMEM;
    } catch (...) {
        if (c) c->err = "internal error";
        return DFT_EINTERNAL;
    }
}

struct Timer {
    cudaEvent_t ev[9];
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        for (auto& e : ev) cudaEventCreate(&e);
    }
    ~Timer() {
        for (auto& e : ev) cudaEventDestroy(e);
    }
    void mark(int i) { cudaEventRecord(ev[i], s); }
    float ms(int a, int b) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) t = 0.f;
        return t;
    }
};

void read_flags(Ctx& c, cudaStream_t s, int* flags) {
    DFT_CUDA_CHECK(cudaMemcpyAsync(flags, c.d_flags, sizeof(int) * FLAG_COUNT, cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
}

// Pulay coefficients: minimise |sum c_i R_i| subject to sum c_i = 1, i.e. the
// bordered system [B -1; -1^T 0][c; l] = [0; -1], by Gaussian elimination
// with partial pivoting; false if singular
bool solve_pulay(int m, const std::vector<double>& B, std::vector<double>* c) {
    int n = m + 1;
    std::vector<double> A((size_t)n * (n + 1), 0.0);
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < m; ++j) A[(size_t)i * (n + 1) + j] = B[(size_t)i * m + j];
        A[(size_t)i * (n + 1) + m] = -1.0;
        A[(size_t)m * (n + 1) + i] = -1.0;
    }
    A[(size_t)m * (n + 1) + n] = -1.0;
    double scale = 0.0;
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(B[(size_t)i * m + i]));
    if (!(scale > 0.0)) return false;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * (n + 1) + col]) > std::fabs(A[(size_t)piv * (n + 1) + col])) piv = r;
        double pv = A[(size_t)piv * (n + 1) + col];
        if (!(std::fabs(pv) > 1e-14 * scale)) return false;
        if (piv != col)
            for (int k = 0; k <= n; ++k) std::swap(A[(size_t)piv * (n + 1) + k], A[(size_t)col * (n + 1) + k]);
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = A[(size_t)r * (n + 1) + col] / pv;
            if (f == 0.0) continue;
            for (int k = col; k <= n; ++k) A[(size_t)r * (n + 1) + k] -= f * A[(size_t)col * (n + 1) + k];
        }
    }
    c->assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        (*c)[i] = A[(size_t)i * (n + 1) + n] / A[(size_t)i * (n + 1) + i];
        if (!std::isfinite((*c)[i])) return false;
    }
    return true;
}

// Pulay (DIIS) mixing, first half: the new history entry (n_in and its
// residual R) goes to ring slot pl_count % H, and one pass over the grids
// writes the new row of B, <R_slot, R_j> for the m filled slots (slots
// 0..m-1), to scal[SCAL_PULAY..] and max|R| to scal[SCAL_RES]
void pulay_begin(Ctx& c, const double* n_in, const double* n_out, cudaStream_t s) {
    const int H = c.pl_hist;
    const int slot = (int)(c.pl_count % H);
    c.pl_count++;
    const int m = (int)std::min<long long>(c.pl_count, H);
    pulay_prepare(c, m, slot, n_in, n_out, c.d_scal + SCAL_PULAY, c.d_scal + SCAL_RES, s);
}

// second half, with the row read back to the host: solve for the
// coefficients and update the input density from the history ring
void pulay_mix(Ctx& c, double* n_in, const double* row_host, cudaStream_t s) {
    const int H = c.pl_hist;
    const int slot = (int)((c.pl_count - 1) % H);
    const int m = (int)std::min<long long>(c.pl_count, H);
    std::vector<double> row(row_host, row_host + m);
    for (int j = 0; j < m; ++j) {
        c.pl_B[(size_t)slot * H + j] = row[j];
        c.pl_B[(size_t)j * H + slot] = row[j];
    }
    // oldest entries are dropped until the system is solvable
    std::vector<int> act;
    for (int k = 0; k < m; ++k) act.push_back((int)((c.pl_count - m + k) % H));
    std::vector<double> coef;
    while (true) {
        int mm = (int)act.size();
        std::vector<double> B((size_t)mm * mm);
        for (int i = 0; i < mm; ++i)
            for (int j = 0; j < mm; ++j) B[(size_t)i * mm + j] = c.pl_B[(size_t)act[i] * H + act[j]];
        if (solve_pulay(mm, B, &coef) || mm == 1) break;
        act.erase(act.begin());
    }
    if (act.size() == 1) coef.assign(1, 1.0);
    std::vector<double> full(H, 0.0);
    for (size_t i = 0; i < act.size(); ++i) full[act[i]] = coef[i];
    DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_scal + SCAL_PULAY + 16, full.data(), sizeof(double) * H,
                                   cudaMemcpyHostToDevice, s));
    pulay_update(c, m, c.d_scal + SCAL_PULAY + 16, n_in, s);
}

// N_C = smallest order whose coefficient tail (at mu = Ebar, the slowest
// decay) sums below tol (the paper's N_C ~ 2 dE beta is the same order)
int auto_order(Ctx& c, double emin, double emax, cudaStream_t s) {
    double de = 0.5 * (emax - emin);
    long long ntry = (long long)std::ceil(12.0 * c.p.beta * de) + 64;
    ntry = std::min<long long>(ntry, c.cheb_cap);
    int M = 4 * (int)ntry;
    launch_cos_table(M, c.d_cos, s);
    launch_cheb_coeffs((int)ntry, M, c.d_cos, c.d_scal, c.p.beta, 0.5 * (emax + emin), true, c.d_coef, s);
    std::vector<double> a(ntry);
    DFT_CUDA_CHECK(cudaMemcpyAsync(a.data(), c.d_coef, sizeof(double) * ntry, cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    double tail = 0.0;
    int nc = (int)ntry;
    for (long long l = ntry - 1; l >= 0; --l) {
        tail += std::fabs(a[l]);
        if (tail >= c.p.cheb_tail_tol) { nc = (int)(l + 1); break; }
        if (l == 0) nc = 1;
    }
    return std::max(nc, 2);
}

// ---- the density matrix in phases (Supp. B); batched SCF steps interleave them ----

// number of moments-pass steps j = 1..J with 2j + 1 <= N_C - 1
inline int pass1_steps(int n_c) { return n_c >= 2 ? (n_c - 2) / 2 : 0; }

// F~ = L^-1 F L^-T, spectral bounds, N_C, H_N, and m_0, m_1, m_2
void dm_prepare(Ctx& c, const double* F, cudaStream_t s, Timer* tm, int t0) {
    if (!c.have_chol) throw Error(DFT_EINVAL, "call dft_overlap_kinetic first");
    const int K = c.K;
    DFT_CUDA_CHECK(cudaMemsetAsync(c.d_flags, 0, sizeof(int) * FLAG_COUNT, s));
    DFT_CUDA_CHECK(cudaMemsetAsync(c.d_scal + SCAL_DMU, 0, sizeof(double) * (SCAL_COUNT - SCAL_DMU), s));
    if (tm) tm->mark(t0);
    // F~ = L^-1 F L^-T: split-FP16 tensor-core products on the mixed path,
    // FP64 on the FP64 path
    if (c.p.precision != DFT_PREC_FP64) cg_transform_f(c, F, c.d_A, s);
    else congruence_lower(K, c.d_Linv, F, c.d_B, c.d_A, s);
    if (tm) tm->mark(t0 + 1);
    if (c.p.e_max > c.p.e_min) {
        double b[2] = {c.p.e_min, c.p.e_max};
        DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_scal + SCAL_EMIN, b, sizeof(b), cudaMemcpyHostToDevice, s));
    } else {
        lanczos_bounds(c, c.d_A, c.p.lanczos_steps > 0 ? c.p.lanczos_steps : 64, s);
    }
    double eb[2];
    DFT_CUDA_CHECK(cudaMemcpyAsync(eb, c.d_scal + SCAL_EMIN, sizeof(eb), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    if (!(eb[1] > eb[0])) throw Error(DFT_ESPECTRUM, "degenerate spectral bounds");
    c.e_bounds[0] = eb[0];
    c.e_bounds[1] = eb[1];
    launch_normalise_h(K, c.d_A, c.d_scal, c.d_H, s);
    int n_c = c.p.cheb_order > 0 ? c.p.cheb_order : auto_order(c, eb[0], eb[1], s);
    if (n_c < 2 || n_c > c.cheb_cap) throw Error(DFT_EINVAL, "Chebyshev order out of range");
    c.n_c_cur = n_c;
    launch_cos_table(4 * n_c, c.d_cos, s);
    if (tm) tm->mark(t0 + 2);
    double m0 = (double)K;
    DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_mom, &m0, sizeof(double), cudaMemcpyHostToDevice, s));
    if (c.p.precision != DFT_PREC_FP64) {
        // split H_N into its 16-bit pair; trace and |H|^2 of the pair
        tc_split_h(c, s);
        tc_init(c, nullptr, s);
        DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_mom + 1, c.d_scal + SCAL_TRACE, sizeof(double), cudaMemcpyDeviceToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_scal + SCAL_TRACE, c.d_scal + SCAL_TRACE + 1, sizeof(double),
                                       cudaMemcpyDeviceToDevice, s));
    } else {
        launch_cheb_init(K, c.d_H, c.d_X0, c.d_X1, nullptr, nullptr, s);
        launch_trace(K, c.d_H, c.d_mom + 1, s);
        launch_frob_dot((long long)K * K, c.d_H, c.d_H, c.d_part, c.d_scal + SCAL_TRACE, s);
    }
    DFT_CUDA_CHECK(cudaMemsetAsync(c.d_scal + SCAL_TRACE + 1, 0, sizeof(double), s));
    if (n_c > 2) launch_moment_reduce(1, c.d_scal + SCAL_TRACE, c.d_mom, 2, -1, m0, c.d_mom + 1, s);
}

// In-flight tuning of the tensor-core launch shape on the weighted pass
// (the dominant one): while the shape of this (precision, size, batch) is
// untuned, the first steps l = 2, 3, ... run each candidate shape on two
// rounds of real steps (two per-step launches, or one dataflow launch of
// eight steps), timed by events, and the fastest per step (minimum over
// rounds) is kept for the rest of the pass and for later calls; no step is
// repeated.  Returns the first step not yet run.
int tc_pass2_tuned(TcBatch& b, int total_k, int Lmax, cudaStream_t s) {
    int l = 2;
    TcCfg cand[12];
    const int nc = tc_candidates(b, cand);
    const int per = 2, per_flow = 8, rounds = 2;
    int need = 0;
    for (int i = 0; i < nc; ++i) need += rounds * (cand[i].flow ? per_flow : per);
    if (tc_needs_tuning(b, total_k) && Lmax - 2 >= need + 8) {
        float best_ms[12];
        for (float& x : best_ms) x = 1e30f;
        cudaEvent_t e0, e1;
        DFT_CUDA_CHECK(cudaEventCreate(&e0));
        DFT_CUDA_CHECK(cudaEventCreate(&e1));
        for (int r = 0; r < rounds; ++r)
            for (int i = 0; i < nc; ++i) {
                b.cfg = cand[i];
                const int n = cand[i].flow ? per_flow : per;
                DFT_CUDA_CHECK(cudaEventRecord(e0, s));
                if (cand[i].flow) {
                    tc_run_flow(b, l, n, 1, 1, s);
                    l += n;
                } else {
                    for (int k = 0; k < n; ++k, ++l) tc_step_batch(b, l, (l + 1) & 1, 1, s);
                }
                DFT_CUDA_CHECK(cudaEventRecord(e1, s));
                DFT_CUDA_CHECK(cudaEventSynchronize(e1));
                float ms = 0.f;
                DFT_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
                best_ms[i] = std::min(best_ms[i], ms / n);
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        int best = 0;
        for (int i = 1; i < nc; ++i)
            if (best_ms[i] < best_ms[best]) best = i;
        tc_record(b, total_k, cand[best], best_ms, nc);
    }
    b.cfg = tc_tuned(b, total_k);
    return l;
}

// moments pass of one system: m_l = Tr T_l(H_N), l < N_C, by doubling
void dm_pass1(Ctx& c, cudaStream_t s) {
    const int K = c.K, n_c = c.n_c_cur, J = pass1_steps(n_c);
    if (c.p.precision != DFT_PREC_FP64) {
        Ctx* cp = &c;
        int lim = J + 1, last = J;
        TcBatch b = tc_batch(c, &cp, 1, &lim, &last, s);
        tc_set_limits(b, &cp, &lim, &last, s);
        b.cfg = tc_tuned(b, K);
        if (b.cfg.flow) {
            tc_run_flow(b, 1, J, 0, 2, s);
            tc_moments_from_fixed(b, J, s);
            return;
        }
        for (int j = 1; j <= J; ++j) {
            tc_step_batch(b, j, j & 1, 2, s);
            tc_moment_reduce_batch(b, j, s);
        }
        return;
    }
    const double m0 = (double)K;
    int nparts = cheb_step_parts(K);
    double* cur = c.d_X1;
    double* prev = c.d_X0;
    for (int j = 1; j <= J; ++j) {
        launch_cheb_step_fp64(K, c.d_H, cur, prev, nullptr, nullptr, 0, c.d_part, c.d_flags, s);
        std::swap(cur, prev);
        launch_moment_reduce(nparts, c.d_part, c.d_mom, (2 * j + 2 < n_c) ? 2 * j + 2 : -1, 2 * j + 1, m0,
                             c.d_mom + 1, s);
    }
}

// mu from 2 sum_l a_l(mu) m_l = N_e (Eq. 2.8), then the coefficients
void dm_mu(Ctx& c, cudaStream_t s) {
    const int n_c = c.n_c_cur, M = 4 * n_c;
    launch_moment_weights(n_c, M, c.d_cos, c.d_mom, c.d_wk, s);
    launch_mu_bisect(M, c.d_cos, c.d_wk, c.p.beta, c.p.n_electrons, c.d_scal, c.d_flags, s);
    launch_cheb_coeffs(n_c, M, c.d_cos, c.d_scal, c.p.beta, 0.0, false, c.d_coef, s);
}

// coefficients a_l(mu) at a given mu (the moments pass skipped), mu on the device
void dm_mu_fixed(Ctx& c, double mu, cudaStream_t s) {
    const int n_c = c.n_c_cur, M = 4 * n_c;
    DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_scal + SCAL_MU, &mu, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_cheb_coeffs(n_c, M, c.d_cos, c.d_scal, c.p.beta, mu, true, c.d_coef, s);
}

// weighted pass of one system: rho = sum_l a_l X_l
void dm_pass2(Ctx& c, cudaStream_t s) {
    const int K = c.K, n_c = c.n_c_cur;
    if (c.p.precision != DFT_PREC_FP64) {
        tc_init(c, c.d_coef, s);
        Ctx* cp = &c;
        int lim = n_c, last = 0;
        TcBatch b = tc_batch(c, &cp, 1, &lim, &last, s);
        tc_set_limits(b, &cp, &lim, &last, s);
        const int l0 = tc_pass2_tuned(b, K, n_c, s);
        if (b.cfg.flow) tc_run_flow(b, l0, n_c - l0, 1, 1, s);
        else
            for (int l = l0; l < n_c; ++l) tc_step_batch(b, l, (l + 1) & 1, 1, s);
        tc_rho_finish(c, s);
        return;
    }
    launch_cheb_init(K, c.d_H, c.d_X0, c.d_X1, c.d_rho, c.d_coef, s);
    double* cur = c.d_X1;
    double* prev = c.d_X0;
    for (int l = 2; l < n_c; ++l) {
        launch_cheb_step_fp64(K, c.d_H, cur, prev, c.d_rho, c.d_coef, l, nullptr, c.d_flags, s);
        std::swap(cur, prev);
    }
}

// P = L^-T rho L^-1, electron count, status flags
// (mixed path: first the FP64 electron-count correction of rho, unless
// switched off; then the split-FP16 tensor-core back-transform)
void dm_finish(Ctx& c, double* P, dft_info* info, cudaStream_t s) {
    const int K = c.K;
    if (c.p.precision != DFT_PREC_FP64) {
        cg_split_rho(c, s);
        if (!c.p.skip_correction) {
            cg_correct_rho(c, s);
            cg_split_rho(c, s);
        }
        cg_back_transform(c, P, s);
    } else {
        congruence_lower_t(K, c.d_Linv, c.d_rho, c.d_B, P, s);
    }
    launch_frob_dot((long long)K * K, P, c.d_S, c.d_part, c.d_scal + SCAL_NE, s);
    int flags[FLAG_COUNT];
    read_flags(c, s, flags);
    double sc[2], corr[4];
    DFT_CUDA_CHECK(cudaMemcpyAsync(sc, c.d_scal + SCAL_MU, sizeof(double), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(sc + 1, c.d_scal + SCAL_NE, sizeof(double), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaMemcpyAsync(corr, c.d_scal + SCAL_DMU, sizeof(corr), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    if (info) {
        info->mu = sc[0];
        info->e_min = c.e_bounds[0];
        info->e_max = c.e_bounds[1];
        info->n_e_trace = 2.0 * sc[1];
        info->n_cheb = c.n_c_cur;
        info->spectrum_ok = flags[FLAG_SPECTRUM] ? 0 : 1;
        info->mu_correction = corr[0];
        info->n_e_uncorrected = corr[1];
        info->e_band_correction = 2.0 * corr[0] * c.p.beta * corr[2];
    }
    c.mu_step_raw = corr[3];
    c.mu_last = sc[0];
    if (flags[FLAG_TIMEOUT]) throw Error(DFT_ETIMEOUT, "a tensor-core pipeline wait expired");
    if (flags[FLAG_RANGE]) throw Error(DFT_EINTERNAL, "a split-precision congruence left the range of the FP16 pair");
    if (flags[FLAG_SPECTRUM]) throw Error(DFT_ESPECTRUM, "Chebyshev iterates left [-1, 1]: spectral bounds too tight");
    if (flags[FLAG_MU]) throw Error(DFT_ENOTCONV, "mu bisection: the bracket does not contain N_e");
}

// P = f(S^-1 F) S^-1 through the symmetric Chebyshev recurrence (Supp. B);
// with mu_fixed the moments pass is skipped and the expansion is taken at
// that mu (the FP64 correction in dm_finish then moves mu to first order)
void density_matrix_impl(Ctx& c, const double* F, double* P, dft_info* info, cudaStream_t s, Timer* tm,
                         int t0, const double* mu_fixed = nullptr) {
    dm_prepare(c, F, s, tm, t0);
    if (mu_fixed) {
        dm_mu_fixed(c, *mu_fixed, s);
    } else {
        dm_pass1(c, s);
        dm_mu(c, s);
    }
    if (tm) tm->mark(t0 + 3);
    dm_pass2(c, s);
    if (tm) tm->mark(t0 + 4);
    dm_finish(c, P, info, s);
    if (tm) tm->mark(t0 + 5);
}

// F += T + V^NL (Eq. 2.3; V^NL only with KB projectors)
void add_one_electron(Ctx& c, double* F, cudaStream_t s) {
    launch_axpby_mat(c.K, 1.0, c.d_T, 1.0, F, F, s);
    if (c.d_VNL) launch_axpby_mat(c.K, 1.0, c.d_VNL, 1.0, F, F, s);
}

// v_KS[n_in] -> V^KS -> F = T + V^NL + V^KS (into c.d_F)
void scf_head(Ctx& c, const double* n_in, cudaStream_t s) {
    hartree_xc(c, n_in, c.d_vks, false, s);
    launch_quadrature(c, c.d_vks, c.d_F, s);
    add_one_electron(c, c.d_F, s);
}

// n_out from c.d_P, energy of n_out, residual, mixing; fills loc
void scf_tail(Ctx& c, double* n_in_out, double* v_ks_out, double* P_out, dft_info* loc, cudaStream_t s, Timer* tm) {
    const int K = c.K;
    if (tm) tm->mark(7);
    launch_collocate(c, c.d_P, c.d_nout, s);
    if (tm) tm->mark(8);
    hartree_xc(c, c.d_nout, nullptr, true, s);
    launch_frob_dot((long long)K * K, c.d_P, c.d_T, c.d_part, c.d_scal + SCAL_EKIN, s);
    if (c.d_VNL) launch_frob_dot((long long)K * K, c.d_P, c.d_VNL, c.d_part, c.d_scal + SCAL_ENL, s);
    if (c.p.mixer == DFT_MIX_PULAY) pulay_begin(c, n_in_out, c.d_nout, s);   // also max|n_out - n_in|
    else launch_maxabs_diff(c.ng, c.d_nout, n_in_out, c.d_part, c.d_scal + SCAL_RES, s);
    if (v_ks_out) DFT_CUDA_CHECK(cudaMemcpyAsync(v_ks_out, c.d_vks, sizeof(double) * c.ng, cudaMemcpyDeviceToDevice, s));
    if (P_out) DFT_CUDA_CHECK(cudaMemcpyAsync(P_out, c.d_P, sizeof(double) * K * K, cudaMemcpyDeviceToDevice, s));
    double sc[SCAL_COUNT];
    DFT_CUDA_CHECK(cudaMemcpyAsync(sc, c.d_scal, sizeof(sc), cudaMemcpyDeviceToHost, s));
    DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    loc->e_kin = 2.0 * sc[SCAL_EKIN];
    loc->e_loc = sc[SCAL_E0];
    loc->e_hartree = sc[SCAL_E1];
    loc->e_xc = sc[SCAL_E2];
    loc->e_nl = c.d_VNL ? 2.0 * sc[SCAL_ENL] : 0.0;
    loc->e_total = loc->e_kin + loc->e_nl + loc->e_loc + loc->e_hartree + loc->e_xc;
    loc->residual = sc[SCAL_RES];
    // mixing (Pulay needs the residual on the host for its small solve)
    if (c.p.mixer == DFT_MIX_KERKER) kerker_mix(c, n_in_out, c.d_nout, c.p.mix_alpha, s);
    else if (c.p.mixer == DFT_MIX_PULAY) pulay_mix(c, n_in_out, sc + SCAL_PULAY, s);
    else launch_linear_mix(c.ng, n_in_out, c.d_nout, c.p.mix_alpha, s);
    loc->de_per_atom = c.have_prev ? (loc->e_total - c.e_prev) / c.n_atoms : 0.0;
    c.e_prev = loc->e_total;
    c.have_prev = true;
    loc->iter = ++c.iter;
    if (tm) loc->ms_stage[6] = tm->ms(7, 8);
}

// Run body(ctx, index, stream) for every system of a batch on host threads,
// each system on its own stream; the systems' streams first wait for the work
// already queued on `s`, and `s` waits for all of them at the end.
template <class F>
void fork_systems(std::vector<Ctx*>& cs, cudaStream_t s, F&& body) {
    const int n = (int)cs.size();
    cudaEvent_t start;
    DFT_CUDA_CHECK(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    DFT_CUDA_CHECK(cudaEventRecord(start, s));
    for (Ctx* c : cs) {
        if (!c->aux_stream) DFT_CUDA_CHECK(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
        if (!c->aux_done) DFT_CUDA_CHECK(cudaEventCreateWithFlags(&c->aux_done, cudaEventDisableTiming));
        DFT_CUDA_CHECK(cudaStreamWaitEvent(c->aux_stream, start, 0));
    }
    int dev = 0;
    DFT_CUDA_CHECK(cudaGetDevice(&dev));
    const int nt = std::min(n, 16);
    std::vector<std::exception_ptr> errs(nt);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t] {
            try {
                DFT_CUDA_CHECK(cudaSetDevice(dev));
                for (int q = t; q < n; q += nt) {
                    body(*cs[q], q, cs[q]->aux_stream);
                    DFT_CUDA_CHECK(cudaEventRecord(cs[q]->aux_done, cs[q]->aux_stream));
                }
            } catch (...) {
                errs[t] = std::current_exception();
            }
        });
    for (auto& x : th) x.join();
    cudaEventDestroy(start);
    for (auto& e : errs)
        if (e) std::rethrow_exception(e);
    for (Ctx* c : cs) DFT_CUDA_CHECK(cudaStreamWaitEvent(s, c->aux_done, 0));
}

// identifies a batch's tile list and launch shape for the graph cache
long long batch_key(const TcBatch& b) {
    long long k = (long long)b.ntiles[0] * 128 + b.nsys;
    k = k * 4 + (b.cfg.bk == 64) + 2 * (b.cfg.bn == 128);
    return (((k * 4 + b.cfg.persist) * 2 + b.cfg.streamk) * 65 + b.cfg.pf) * 2 + b.cfg.epf;
}

// run a launch sequence through a CUDA graph cached in `lead` under (slot,
// count): the recurrence loops are thousands of launches that repeat
// unchanged from one SCF step to the next while N_C stays the same
template <class F>
void run_graph(Ctx& lead, int slot, int count, long long key, cudaStream_t s, F&& body) {
    if (count <= 0) return;
    if (!lead.graph_exec[slot] || lead.graph_count[slot] != count || lead.graph_key[slot] != key) {
        if (lead.graph_exec[slot]) {
            cudaGraphExecDestroy(lead.graph_exec[slot]);
            lead.graph_exec[slot] = nullptr;
        }
        cudaStream_t cs = nullptr;
        DFT_CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        DFT_CUDA_CHECK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            body(cs);
        } catch (...) {
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cs);
            throw;
        }
        DFT_CUDA_CHECK(cudaStreamEndCapture(cs, &g));
        cudaError_t e = cudaGraphInstantiate(&lead.graph_exec[slot], g, 0);
        cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) throw Error(DFT_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        lead.graph_count[slot] = count;
        lead.graph_key[slot] = key;
    }
    DFT_CUDA_CHECK(cudaGraphLaunch(lead.graph_exec[slot], s));
}

}  // namespace

extern "C" {

const char* dft_version(void) { return kVersion; }

unsigned long long dft_kernel_launches(void) { return g_launches.load(); }

size_t dft_workspace_bytes(const dft_basis_desc* basis, const dft_grid_desc* grid, const dft_params* params) {
    try {
        validate(basis, grid, params);
        Ctx c;
        build_basis(c, basis, grid, params, nullptr, nullptr);
        return carve(c, nullptr);
    } catch (...) {
        return 0;
    }
}

dft_status dft_init_basis(dft_ctx** ctx, const dft_basis_desc* basis, const dft_grid_desc* grid,
                          const dft_params* params, void* workspace, size_t ws_bytes, void* stream) {
    if (!ctx) return DFT_EINVAL;
    *ctx = nullptr;
    Ctx* c = new (std::nothrow) Ctx();
    if (!c) return DFT_ENOMEM;
    dft_status st = guarded(reinterpret_cast<dft_ctx*>(c), [&] {
        validate(basis, grid, params);
        if (!workspace) throw Error(DFT_EINVAL, "null workspace");
        if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) throw Error(DFT_EINVAL, "workspace must be 256-byte aligned");
        std::vector<int> tp, tf;
        build_basis(*c, basis, grid, params, &tp, &tf);
        size_t need = carve(*c, nullptr);
        if (ws_bytes < need) throw Error(DFT_ENOMEM, "workspace too small: need " + std::to_string(need) + " bytes");
        carve(*c, static_cast<char*>(workspace));
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_fn, c->fn_host.data(), sizeof(Fn) * c->Kt, cudaMemcpyHostToDevice, s));
        if (c->contracted) {
            std::vector<int> par(c->Kt);
            for (int a = 0; a < c->K; ++a)
                for (int t = c->term_ptr_host[a]; t < c->term_ptr_host[a + 1]; ++t) par[t] = a;
            DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_term_ptr, c->term_ptr_host.data(), sizeof(int) * (c->K + 1),
                                           cudaMemcpyHostToDevice, s));
            DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_term_par, par.data(), sizeof(int) * c->Kt, cudaMemcpyHostToDevice, s));
        }
        DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_tile_ptr, tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice, s));
        if (!tf.empty())
            DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_tile_fn, tf.data(), sizeof(int) * tf.size(), cudaMemcpyHostToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_xyz, c->xyz_host.data(), sizeof(double) * c->xyz_host.size(),
                                       cudaMemcpyHostToDevice, s));
        if (!c->pj_host.empty()) {
            DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_pj, c->pj_host.data(), sizeof(Fn) * c->pj_host.size(),
                                           cudaMemcpyHostToDevice, s));
            DFT_CUDA_CHECK(cudaMemcpyAsync(c->d_pje, c->pje_host.data(), sizeof(double) * c->pje_host.size(),
                                           cudaMemcpyHostToDevice, s));
        }
        DFT_CUDA_CHECK(cudaMemsetAsync(c->d_scal, 0, sizeof(double) * SCAL_COUNT, s));
        DFT_CUDA_CHECK(cudaMemsetAsync(c->d_flags, 0, sizeof(int) * FLAG_COUNT, s));
        if (c->Kp > 0) {
            DFT_CUDA_CHECK(cudaMemsetAsync(c->d_x16[0], 0, (size_t)c->Kp * c->Kp * 2 * 4, s));
            tc_setup(*c);
            cg_setup(*c);
        }
        launch_build_tables(*c, s);
        if (c->contracted) {
            // the functions' normalisation N_a from the closed-form overlap of
            // their terms (needed by every contraction and expansion)
            launch_overlap_kinetic_terms(*c, c->d_Mt, s);
            launch_contract_norms(*c, c->d_Mt, s);
        }
        launch_gaussian_sum(*c, -c->p.vloc_depth, c->p.vloc_width, c->d_vloc, s);
        double w = c->p.vloc_width;
        launch_gaussian_sum(*c, c->p.ion_charge * std::pow(M_PI * w * w, -1.5), w, c->d_nion, s);
        poisson_setup(*c, s);
        if (c->p.mixer == DFT_MIX_KERKER || (c->p.mixer == DFT_MIX_PULAY && c->p.kerker_q0 > 0.0))
            kerker_setup(*c, s);
        c->pl_B.assign((size_t)c->pl_hist * c->pl_hist, 0.0);
        DFT_CUDA_CHECK(cudaStreamSynchronize(s));
    });
    if (st != DFT_OK) {
        // keep the context so the caller can read the message, but mark it unusable
        c->K = 0;
        *ctx = reinterpret_cast<dft_ctx*>(c);
        return st;
    }
    *ctx = reinterpret_cast<dft_ctx*>(c);
    return DFT_OK;
}

dft_status dft_overlap_kinetic(dft_ctx* ctx, double* S, double* T, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0) throw Error(DFT_EINVAL, "context not initialised");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        size_t K2 = sizeof(double) * (size_t)c.K * c.K;
        launch_overlap_kinetic(c, c.d_S, c.d_T, s);
        if (S) DFT_CUDA_CHECK(cudaMemcpyAsync(S, c.d_S, K2, cudaMemcpyDeviceToDevice, s));
        if (T) DFT_CUDA_CHECK(cudaMemcpyAsync(T, c.d_T, K2, cudaMemcpyDeviceToDevice, s));
        DFT_CUDA_CHECK(cudaMemcpyAsync(c.d_A, c.d_S, K2, cudaMemcpyDeviceToDevice, s));
        DFT_CUDA_CHECK(cudaMemsetAsync(c.d_flags, 0, sizeof(int) * FLAG_COUNT, s));
        cholesky_inplace(c.d_A, c.K, c.d_flags + FLAG_CHOL, s);
        c.mu_count = 0;   // a new geometry: no settled chemical potential yet
        tri_inverse_lower(c.d_A, c.d_Linv, c.K, c.d_B, s);
        if (c.Kp > 0) cg_split_linv(c, s);   // L^-1, L^-T as FP16 pairs for the mixed congruences
        if (c.d_VNL) launch_nonlocal(c, s);  // V^NL, once per geometry (Supp. A.2.2)
        int flags[FLAG_COUNT];
        read_flags(c, s, flags);
        if (flags[FLAG_CHOL]) throw Error(DFT_ENOTCONV, "overlap matrix is not positive definite");
        if (flags[FLAG_RANGE]) throw Error(DFT_EINTERNAL, "L^-1 is outside the range of the FP16 pair");
        c.have_chol = true;
    });
}

dft_status dft_density_matrix_columns(dft_ctx* ctx, const double* F, const int* cols, int ncols, double mu,
                                      double e_min, double e_max, int n_cheb, double thresh, int precond,
                                      double pcg_tol, int pcg_maxit, double* out, dft_columns_info* info,
                                      void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !F || !cols || !out) throw Error(DFT_EINVAL, "null argument");
        if (!c.have_chol) throw Error(DFT_EINVAL, "call dft_overlap_kinetic first");
        // 32-bit CSR row offsets: at most K^2 kept entries must stay below 2^31
        if ((long long)c.K * c.K > 2147483647LL) throw Error(DFT_EINVAL, "K too large for 32-bit CSR offsets");
        if (ncols < 1) throw Error(DFT_EINVAL, "ncols must be positive");
        for (int i = 0; i < ncols; ++i)
            if (cols[i] < 0 || cols[i] >= c.K) throw Error(DFT_EINVAL, "column index outside [0, K)");
        if (n_cheb < 2 || n_cheb > c.cheb_cap) throw Error(DFT_EINVAL, "n_cheb outside [2, Chebyshev capacity]");
        if (!(e_max > e_min) || !std::isfinite(e_min) || !std::isfinite(e_max) || !std::isfinite(mu))
            throw Error(DFT_EINVAL, "need finite mu and e_min < e_max");
        if (!(thresh >= 0.0)) throw Error(DFT_EINVAL, "thresh must be >= 0");
        if (!(pcg_tol > 0.0) || pcg_maxit < 1) throw Error(DFT_EINVAL, "need pcg_tol > 0 and pcg_maxit >= 1");
        if (precond != DFT_PRECOND_BLOCK_JACOBI && precond != DFT_PRECOND_NONE)
            throw Error(DFT_EINVAL, "unknown preconditioner");
        require_aligned16({F, out});
        sparse_columns(c, F, cols, ncols, mu, e_min, e_max, n_cheb, thresh, precond, pcg_tol, pcg_maxit, out, info,
                       static_cast<cudaStream_t>(stream));
    });
}

dft_status dft_nonlocal_matrix(dft_ctx* ctx, double* VNL, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !VNL) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({VNL});
        if (!c.have_chol) throw Error(DFT_EINVAL, "call dft_overlap_kinetic first");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const size_t K2 = sizeof(double) * (size_t)c.K * c.K;
        if (c.d_VNL) DFT_CUDA_CHECK(cudaMemcpyAsync(VNL, c.d_VNL, K2, cudaMemcpyDeviceToDevice, s));
        else DFT_CUDA_CHECK(cudaMemsetAsync(VNL, 0, K2, s));
    });
}

dft_status dft_density_matrix(dft_ctx* ctx, const double* F, double* P, dft_info* info, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !F || !P) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({F, P});
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        Timer tm(s);
        density_matrix_impl(c, F, P, info, s, &tm, 0);
        if (info) {
            std::memset(info->ms_stage, 0, sizeof(info->ms_stage));
            for (int i = 0; i < 5; ++i) info->ms_stage[1 + i] = tm.ms(i, i + 1);
        }
    });
}

dft_status dft_density_on_grid(dft_ctx* ctx, const double* P, double* n_grid, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !P || !n_grid) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({P, n_grid});
        launch_collocate(c, P, n_grid, static_cast<cudaStream_t>(stream));
    });
}

dft_status dft_potential_matrix(dft_ctx* ctx, const double* v_grid, double* V, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !v_grid || !V) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({v_grid, V});
        launch_quadrature(c, v_grid, V, static_cast<cudaStream_t>(stream));
    });
}

dft_status dft_hartree_xc(dft_ctx* ctx, const double* n_grid, double* v_ks, double* energies, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !n_grid) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({n_grid, v_ks});
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        hartree_xc(c, n_grid, v_ks, energies != nullptr, s);
        if (energies) {
            DFT_CUDA_CHECK(cudaMemcpyAsync(energies, c.d_scal + SCAL_E0, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            DFT_CUDA_CHECK(cudaStreamSynchronize(s));
        }
    });
}

dft_status dft_initial_density(dft_ctx* ctx, double* n_grid, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !n_grid) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({n_grid});
        double w = c.p.vloc_width;
        launch_gaussian_sum(c, c.p.ion_charge * std::pow(M_PI * w * w, -1.5), w, n_grid,
                            static_cast<cudaStream_t>(stream));
    });
}

dft_status dft_scf_step(dft_ctx* ctx, double* n_in_out, double* v_ks_out, double* P_out, dft_info* info,
                        void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !n_in_out) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({n_in_out, v_ks_out, P_out});
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        Timer tm(s);
        dft_info loc{};
        tm.mark(0);
        scf_head(c, n_in_out, s);
        tm.mark(1);
        // Skip the moments pass while mu has settled: the last two cycles'
        // chemical potentials within MU_SETTLED kT.  The expansion is then taken
        // at the last mu and the FP64 correction moves mu to first order; a
        // Newton step beyond MU_REDO kT (first-order error no longer small, or
        // no states at the Fermi level) runs the cycle's density matrix again
        // with the moments pass.
        const bool reuse = c.p.reuse_mu && c.p.precision != DFT_PREC_FP64 && !c.p.skip_correction &&
                           c.mu_count >= 2 && std::fabs(c.p.beta * (c.mu_hist[0] - c.mu_hist[1])) < MU_SETTLED;
        if (reuse) {
            const double mu0 = c.mu_hist[0];
            density_matrix_impl(c, c.d_F, c.d_P, &loc, s, &tm, 1, &mu0);
            loc.mu_reused = 1;
            if (!(std::fabs(c.p.beta * c.mu_step_raw) <= MU_REDO)) {
                density_matrix_impl(c, c.d_F, c.d_P, &loc, s, &tm, 1);
                loc.mu_reused = 0;
            }
        } else {
            density_matrix_impl(c, c.d_F, c.d_P, &loc, s, &tm, 1);
        }
        c.mu_hist[1] = c.mu_hist[0];
        c.mu_hist[0] = c.mu_last;
        c.mu_count++;
        scf_tail(c, n_in_out, v_ks_out, P_out, &loc, s, &tm);
        loc.ms_stage[0] = tm.ms(0, 1);
        for (int i = 1; i < 6; ++i) loc.ms_stage[i] = tm.ms(i, i + 1);
        if (info) *info = loc;
    });
}

dft_status dft_scf_step_batched(dft_ctx* const* ctxs, int n, double* const* n_in_out, dft_info* infos,
                                void* stream) {
    if (!ctxs || n < 1 || !ctxs[0]) return DFT_EINVAL;
    return guarded(ctxs[0], [&] {
        if (n > TC_MAX_SYS) throw Error(DFT_EINVAL, "at most 64 systems per batch");
        if (!n_in_out) throw Error(DFT_EINVAL, "null argument");
        std::vector<Ctx*> cs(n);
        for (int q = 0; q < n; ++q) {
            if (!ctxs[q] || !n_in_out[q]) throw Error(DFT_EINVAL, "null context or density in the batch");
            require_aligned16({n_in_out[q]});
            cs[q] = reinterpret_cast<Ctx*>(ctxs[q]);
            if (cs[q]->K == 0 || cs[q]->Kp == 0) throw Error(DFT_EINVAL, "batched steps need mixed-precision contexts");
            if (cs[q]->p.precision != cs[0]->p.precision) throw Error(DFT_EINVAL, "batch mixes precisions");
            for (int r = 0; r < q; ++r)
                if (cs[r] == cs[q]) throw Error(DFT_EINVAL, "a context appears twice in the batch");
        }
        Ctx& lead = *cs[0];
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        Timer tm(s);
        std::vector<dft_info> loc(n);
        tm.mark(0);
        // per system, concurrently on the systems' own streams: potential, Fock
        // matrix, bounds, N_C, split H_N, m_0..m_2 (each waits on the host for
        // its bounds and order, so systems overlap each other's waits)
        fork_systems(cs, s, [&](Ctx& c, int q, cudaStream_t as) {
            scf_head(c, n_in_out[q], as);
            dm_prepare(c, c.d_F, as, nullptr, 0);
        });
        tm.mark(1);
        // moments pass over all systems: one dataflow launch, or one launch per
        // step replayed from a CUDA graph
        std::vector<int> lim(n), last(n);
        int Jmax = 0, Lmax = 0;
        for (int q = 0; q < n; ++q) {
            int J = pass1_steps(cs[q]->n_c_cur);
            lim[q] = J + 1;
            last[q] = J;
            Jmax = std::max(Jmax, J);
            Lmax = std::max(Lmax, cs[q]->n_c_cur);
        }
        TcBatch b = tc_batch(lead, cs.data(), n, lim.data(), last.data(), s);
        tc_set_limits(b, cs.data(), lim.data(), last.data(), s);
        int total_k = 0;
        for (int q = 0; q < n; ++q) total_k += cs[q]->K;
        b.cfg = tc_tuned(b, total_k);
        const long long gkey1 = batch_key(b);
        if (b.cfg.flow) {
            tc_run_flow(b, 1, Jmax, 0, 2, s);
            tc_moments_from_fixed(b, Jmax, s);
        } else {
            run_graph(lead, 0, Jmax, gkey1, s, [&](cudaStream_t gs) {
                for (int j = 1; j <= Jmax; ++j) {
                    tc_step_batch(b, j, j & 1, 2, gs);
                    tc_moment_reduce_batch(b, j, gs);
                }
            });
        }
        tm.mark(2);
        for (int q = 0; q < n; ++q) {
            dm_mu(*cs[q], s);
            tc_init(*cs[q], cs[q]->d_coef, s);
            lim[q] = cs[q]->n_c_cur;
            last[q] = 0;
        }
        tc_set_limits(b, cs.data(), lim.data(), last.data(), s);
        tm.mark(3);
        const int l0 = tc_pass2_tuned(b, total_k, Lmax, s);
        const long long gkey2 = batch_key(b) * 65536 + l0;
        if (b.cfg.flow) {
            tc_run_flow(b, l0, Lmax - l0, 1, 1, s);
        } else {
            run_graph(lead, 1, Lmax - l0, gkey2, s, [&](cudaStream_t gs) {
                for (int l = l0; l < Lmax; ++l) tc_step_batch(b, l, (l + 1) & 1, 1, gs);
            });
        }
        tm.mark(4);
        fork_systems(cs, s, [&](Ctx& c, int q, cudaStream_t as) {
            tc_rho_finish(c, as);
            dm_finish(c, c.d_P, &loc[q], as);
            c.mu_hist[1] = c.mu_hist[0];
            c.mu_hist[0] = c.mu_last;
            c.mu_count++;
            scf_tail(c, n_in_out[q], nullptr, nullptr, &loc[q], as, nullptr);
        });
        tm.mark(5);
        for (int q = 0; q < n; ++q) {
            loc[q].ms_stage[0] = tm.ms(0, 1);   // shared stages: potentials, Fock, bounds (all systems)
            loc[q].ms_stage[3] = tm.ms(1, 2);   // joint moments pass
            loc[q].ms_stage[4] = tm.ms(3, 4);   // joint Chebyshev pass
            loc[q].ms_stage[5] = tm.ms(4, 5);   // back-transforms, collocation, energies, mixing
            if (infos) infos[q] = loc[q];
        }
    });
}

dft_status dft_destroy(dft_ctx* ctx) {
    if (!ctx) return DFT_OK;
    Ctx* c = reinterpret_cast<Ctx*>(ctx);
    for (auto& g : c->graph_exec)
        if (g) cudaGraphExecDestroy(g);
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    if (c->aux_done) cudaEventDestroy(c->aux_done);
    if (c->plan_f) cufftDestroy(c->plan_f);
    if (c->plan_b) cufftDestroy(c->plan_b);
    if (c->kplan_f) cufftDestroy(c->kplan_f);
    if (c->kplan_b) cufftDestroy(c->kplan_b);
    delete c;
    return DFT_OK;
}

dft_status dft_density_from_potential(dft_ctx* ctx, const double* v_grid, double* n_out, dft_info* info,
                                      void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !v_grid || !n_out) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({v_grid, n_out});
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        launch_quadrature(c, v_grid, c.d_F, s);
        add_one_electron(c, c.d_F, s);
        dft_info loc{};
        density_matrix_impl(c, c.d_F, c.d_P, &loc, s, nullptr, 0);
        launch_collocate(c, c.d_P, n_out, s);
        if (info) *info = loc;
    });
}

size_t dft_warmstart_state_bytes(void) { return warm_state_bytes(); }

int dft_warmstart_param_count(void) { return warm_nparam(); }

dft_status dft_warmstart_init(void* state, const float* params, void* stream) {
    if (!state) return DFT_EINVAL;
    try {
        warm_init(state, params, static_cast<cudaStream_t>(stream));
        return DFT_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

dft_status dft_warmstart_potential(dft_ctx* ctx, const void* state, const double* v_start, double* v0,
                                   void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !state || !v0) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({state, v_start, v0});
        warm_forward(c, state, v_start, v0, false, static_cast<cudaStream_t>(stream));
    });
}

dft_status dft_warmstart_accumulate(dft_ctx* ctx, void* state, const double* v_start, const double* v_target,
                                    double* loss, void* stream) {
    if (!ctx) return DFT_EINVAL;
    return guarded(ctx, [&] {
        Ctx& c = *reinterpret_cast<Ctx*>(ctx);
        if (c.K == 0 || !state || !v_target) throw Error(DFT_EINVAL, "null argument");
        require_aligned16({state, v_start, v_target});
        double L = warm_accumulate(c, state, v_start, v_target, static_cast<cudaStream_t>(stream));
        if (loss) *loss = L;
    });
}

dft_status dft_warmstart_adam(void* state, float lr, int step, void* stream) {
    if (!state || step < 1) return DFT_EINVAL;
    try {
        warm_adam(state, lr, step, static_cast<cudaStream_t>(stream));
        return DFT_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

dft_status dft_warmstart_read(const void* state, float* params, float* grads, void* stream) {
    if (!state) return DFT_EINVAL;
    try {
        if (params) warm_params(state, params, static_cast<cudaStream_t>(stream));
        if (grads) warm_grad(state, grads, static_cast<cudaStream_t>(stream));
        return DFT_OK;
    } catch (const Error& e) {
        return e.code;
    }
}

const char* dft_last_error(const dft_ctx* ctx) {
    if (!ctx) return "null context";
    return reinterpret_cast<const Ctx*>(ctx)->err.c_str();
}

}  // extern "C"
