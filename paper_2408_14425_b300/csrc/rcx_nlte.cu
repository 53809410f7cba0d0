// rcx_nlte.cu -- the non-LTE population update around the formal solution (Sec. 3.3):
// model atom tables, LTE start, line opacity/emissivity from populations, statistical
// equilibrium with MALI rates of a diagonal operator, and the iteration driver.
//
// Precision: populations, temperatures and densities are FP64; the profile sums, the
// rates, the rate matrix and its solve are FP64 as well (one thread per cell, a few
// hundred FP64 operations -- negligible next to the formal solution); chi/eta handed to
// the FP32 formal solution and the J_eff / (1 - Lambda*) it returns are FP32.
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rcx_internal.h"

namespace {

// CODATA 2018
constexpr double kH = 6.62607015e-34;
constexpr double kC = 2.99792458e8;
constexpr double kK = 1.380649e-23;
constexpr double kEV = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kAmu = 1.66053906660e-27;
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kRydbergE = 13.605693122994 * kEV;   // van Regemorter's E_H
constexpr double kChiH = 13.598434599702 * kEV;       // hydrogen ionisation energy
constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;

constexpr int kMaxLevels = 8;
constexpr int kMaxLines = 16;
constexpr int kMaxPerLine = 64;

struct LineConst {
    int lo, up, lam0;
    double A, Blu, Bul;
    double hnu_4pi;      // h nu0 / 4 pi
    double dop;          // Doppler width / sqrt(T): nu0/c sqrt(2 k / m)
    double coll;         // n_e-independent van Regemorter factor: beta Omega/(g_l P) = beta (8pi/sqrt3)(E_Ryd/dE) f_lu
    double y_T;          // dE / k: y = y_T / T
    double glo_gup;      // g_l / g_u
    double ddnu;         // frequency step of the line's grid (Hz); the grid is uniform and
                         // symmetric about nu0
};

struct AtomDev {
    int n_levels, n_lines, n_per_line;
    double E_k[kMaxLevels];   // E / k  (K)
    double g[kMaxLevels];
    LineConst line[kMaxLines];
    const double* dnu;        // [n_lines][n_per_line]: nu_k - nu0
    const double* w;          // [n_lines][n_per_line]: trapezoid weights (Hz)
};

rc_status nfail(rc_status s, const std::string& m) {
    rcx::set_last_error(m);
    return s;
}
rc_status ncuda(cudaError_t e, const char* what) {
    cudaGetLastError();
    rcx::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
    return RC_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// 1 / (k k!), the coefficient of (-y)^k in the power series of E1 (evaluated at compile time)
__host__ __device__ constexpr double e1_coef(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return 1.0 / ((double)k * f);
}

// sum_{k=K..N} (-y)^(k-K) / (k k!) by Horner's rule in z = -y (FMAs only: FP64 divisions are
// an order of magnitude dearer than FMAs, and this runs for every line of every hot cell)
template <int K, int N>
__device__ __forceinline__ double e1_horner(double z) {
    constexpr double c = e1_coef(K);
    if constexpr (K == N) return c;
    else return fma(e1_horner<K + 1, N>(z), z, c);
}

// e^y E1(y) through the power series of E1 (Abramowitz & Stegun 5.1.11) for y < 1:
// E1(y) = -gamma - ln y - sum_{k>=1} (-y)^k / (k k!), 30 terms (the 30th is below 1e-33).
__device__ double exp_e1_small(double y) {
    const double z = -y;
    const double sum = z * e1_horner<1, 30>(z);
    return exp(y) * (-kEulerGamma - log(y) - sum);
}

// van Regemorter's effective Gaunt factor P(y) = max(0.2, 0.276 e^y E1(y)); for y >= 1,
// e^y E1(y) <= 0.597 so the floor 0.2 applies.
__device__ double van_regemorter_p(double y) {
    if (y >= 1.0) return 0.2;
    return fmax(0.2, 0.276 * exp_e1_small(y));
}

// The Gaussian exp(-(dnu_k / dD)^2) on a line's uniform grid symmetric about nu0, walked
// from the centre outwards: with offsets u_j = (j + d) h (h = step / dD, d = 0 for an odd
// point count, 1/2 for an even one), e_{j+1} = e_j r_j and r_{j+1} = r_j exp(-2 h^2), so
// one exponential per line replaces one per point (FP64 exponentials are the cost of
// these kernels): for an odd count r_0 = exp(-h^2) and exp(-2 h^2) = r_0^2; for an even one
// e_0 = exp(-h^2 / 4) and r_0 = exp(-2 h^2) = e_0^8.  After j products the relative error
// is a few j ulps.  Calls f(k, e_k) for every grid index k.
template <class F>
__device__ __forceinline__ void for_each_gauss(int n, double h, F&& f) {
    const bool odd = n & 1;
    double e, r, q;
    if (odd) {
        e = 1.0;                                          // e_0 = exp(0)
        r = exp(-h * h);                                  // e_1 / e_0 = exp(-h^2)
        q = r * r;                                        // exp(-2 h^2)
    } else {
        e = exp(-0.25 * h * h);                           // e_0 = exp(-(h / 2)^2)
        const double e2 = e * e, e4 = e2 * e2;
        r = e4 * e4;                                      // e_1 / e_0 = exp(-2 h^2)
        q = r;
    }
    const int hi = n / 2, lo = odd ? n / 2 : n / 2 - 1;    // the centre point(s)
    for (int j = 0; hi + j < n; ++j) {
        f(hi + j, e);
        if (lo - j != hi + j) f(lo - j, e);
        e *= r;
        r *= q;
    }
}

__global__ void lte_kernel(AtomDev A, const double* __restrict__ T, const double* __restrict__ nH,
                           long long ncell, double saha_c, double chi_k, double* __restrict__ ne,
                           double* __restrict__ n_atom, double* __restrict__ pops) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double t = T[c], n = nH[c];
    // x^2 n / (1 - x) = phi with phi = (2 pi m_e k T / h^2)^1.5 exp(-chi_H / kT)
    const double phi = saha_c * t * sqrt(t) * exp(-chi_k / t);
    const double s = sqrt(phi * phi + 4.0 * n * phi);
    const double x = 2.0 * phi / (phi + s);
    const double na = n * (4.0 * n * phi / ((phi + s) * (phi + s)));  // n (1 - x)
    ne[c] = x * n;
    n_atom[c] = na;
    double b[kMaxLevels], sum = 0.0;
    for (int i = 0; i < A.n_levels; ++i) {
        b[i] = A.g[i] * exp(-A.E_k[i] / t);
        sum += b[i];
    }
    for (int i = 0; i < A.n_levels; ++i) pops[(size_t)i * ncell + c] = na * b[i] / sum;
}

__global__ void emis_opac_kernel(AtomDev A, const double* __restrict__ T,
                                 const double* __restrict__ pops, long long ncell,
                                 float* __restrict__ chi, float* __restrict__ eta) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const double sqT = sqrt(T[c]);
    for (int li = 0; li < A.n_lines; ++li) {
        const LineConst& L = A.line[li];
        const double h = L.ddnu / (L.dop * sqT);
        const double* w = A.w + (size_t)li * A.n_per_line;
        double norm = 0.0;
        for_each_gauss(A.n_per_line, h, [&](int k, double g) { norm += w[k] * g; });
        const double nl = pops[(size_t)L.lo * ncell + c], nu = pops[(size_t)L.up * ncell + c];
        // phi_k = gauss / (sqrt(pi) dD) renormalised: the sqrt(pi) dD cancels
        const double kchi = L.hnu_4pi * (nl * L.Blu - nu * L.Bul) / norm;
        const double keta = L.hnu_4pi * nu * L.A / norm;
        for_each_gauss(A.n_per_line, h, [&](int k, double g) {
            const size_t o = (size_t)(L.lam0 + k) * ncell + c;
            chi[o] = (float)(kchi * g);
            eta[o] = (float)(keta * g);
        });
    }
}

// Gamma n = 0 for cell c (Eq. 20) from the per-line integrals Jb[li] = sum_k w phi J_eff and
// Lc[li] = sum_k w phi (1 - Lambda*) (MALI rates, Sec. 3.3) and the collisions; the most
// populated level's row replaced by sum n = n_atom; FP64 throughout.  Writes the new
// populations and returns max |n_new - n_old| / n_new (infinite for a NaN).
__device__ double solve_cell(const AtomDev& A, long long c, long long ncell, double t, double nec,
                             double na, const double* Jb, const double* Lc,
                             double* __restrict__ pops) {
    const int n = A.n_levels;
    const double sqT = sqrt(t);
    double G[kMaxLevels][kMaxLevels];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) G[i][j] = 0.0;
    for (int li = 0; li < A.n_lines; ++li) {
        const LineConst& L = A.line[li];
        const double Rlu = L.Blu * Jb[li];
        const double Rul = L.A * Lc[li] + L.Bul * Jb[li];
        const double y = L.y_T / t;
        // detailed balance: C_ul = C_lu (g_l / g_u) e^{y}, so the common factor carries no
        // exponential and C_ul needs none
        const double base = nec * L.coll * van_regemorter_p(y) / sqT;
        const double Clu = base * exp(-y);
        const double Cul = base * L.glo_gup;
        G[L.up][L.lo] += Rlu + Clu;                  // lo -> up, per atom in lo
        G[L.lo][L.up] += Rul + Cul;                  // up -> lo, per atom in up
    }
    double old[kMaxLevels];
    int r = 0;
    for (int i = 0; i < n; ++i) {
        old[i] = pops[(size_t)i * ncell + c];
        if (old[i] > old[r]) r = i;
    }
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            if (i != j) s += G[i][j];
        G[j][j] = -s;
    }
    double b[kMaxLevels];
    for (int i = 0; i < n; ++i) b[i] = 0.0;
    for (int j = 0; j < n; ++j) G[r][j] = 1.0;       // particle conservation
    b[r] = na;
    // Gaussian elimination with partial pivoting
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(G[i][col]) > fabs(G[p][col])) p = i;
        if (p != col) {
            for (int j = 0; j < n; ++j) {
                const double tmp = G[col][j];
                G[col][j] = G[p][j];
                G[p][j] = tmp;
            }
            const double tb = b[col];
            b[col] = b[p];
            b[p] = tb;
        }
        const double inv = 1.0 / G[col][col];
        for (int i = col + 1; i < n; ++i) {
            const double f = G[i][col] * inv;
            if (f == 0.0) continue;
            for (int j = col; j < n; ++j) G[i][j] -= f * G[col][j];
            b[i] -= f * b[col];
        }
    }
    double x[kMaxLevels];
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= G[i][j] * x[j];
        x[i] = s / G[i][i];
    }
    double rel = 0.0;
    for (int i = 0; i < n; ++i) {
        pops[(size_t)i * ncell + c] = x[i];
        const double d = fabs(x[i] - old[i]) / fabs(x[i]);
        rel = (d == d) ? fmax(rel, d) : INFINITY;    // NaN -> infinite change
    }
    return rel;
}

// block max of a non-negative double -> one atomic per block (non-negative doubles order like
// their bits)
__device__ __forceinline__ void block_max_to(double rel, unsigned long long* dmax_bits) {
    __shared__ double red[256];
    red[threadIdx.x] = rel;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0 && dmax_bits)
        atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(red[0]));
}

// The line integrals of cell c over the grid wavelengths [lam_begin, lam_begin + lam_count) of
// every line (J_eff, alo_c hold those wavelengths only, [lam - lam_begin][cell]); the profile
// is normalised over the whole line, so integrals over disjoint wavelength ranges add up to the
// integral over the line.  alo_c NULL means Lambda* = 0.
__device__ __forceinline__ void line_integrals_cell(const AtomDev& A, long long c, long long ncell,
                                                    double t, const float* __restrict__ Jeff,
                                                    const float* __restrict__ aloc, int lam_begin,
                                                    int lam_count, double* Jb, double* Lc) {
    const double sqT = sqrt(t);
    for (int li = 0; li < A.n_lines; ++li) {
        const LineConst& L = A.line[li];
        const double h = L.ddnu / (L.dop * sqT);
        const double* w = A.w + (size_t)li * A.n_per_line;
        double norm = 0.0, sj = 0.0, sl = 0.0;
        for_each_gauss(A.n_per_line, h, [&](int k, double g) {
            const double wp = w[k] * g;
            norm += wp;
            const int lam = L.lam0 + k - lam_begin;
            if (lam >= 0 && lam < lam_count) {
                const size_t o = (size_t)lam * ncell + c;
                sj += wp * (double)Jeff[o];
                sl += aloc ? wp * (double)aloc[o] : wp;
            }
        });
        Jb[li] = sj / norm;                 // sum_k w phi J_eff
        Lc[li] = sl / norm;                 // sum_k w phi (1 - Lambda*)
    }
}

// Gamma n = 0 per cell (Eq. 20) with MALI rates from J_eff and 1 - Lambda* of every wavelength.
__global__ void stat_eq_kernel(AtomDev A, const double* __restrict__ T,
                               const double* __restrict__ ne, const double* __restrict__ n_atom,
                               const float* __restrict__ Jeff, const float* __restrict__ aloc,
                               long long ncell, double* __restrict__ pops,
                               unsigned long long* __restrict__ dmax_bits,
                               const unsigned char* __restrict__ active) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    // cells outside a sparse plan's active set (Sec. 3.5) keep their populations
    if (c < ncell && (!active || active[c])) {
        double Jb[kMaxLines], Lc[kMaxLines];
        line_integrals_cell(A, c, ncell, T[c], Jeff, aloc, 0, 1 << 30, Jb, Lc);
        rel = solve_cell(A, c, ncell, T[c], ne[c], n_atom[c], Jb, Lc, pops);
    }
    block_max_to(rel, dmax_bits);
}

// Partial line integrals over a range of the atom's wavelengths: out [line][2][cell] =
// (sum_k w phi J_eff, sum_k w phi (1 - Lambda*)) over the range's grid points.
__global__ void line_integrals_kernel(AtomDev A, const double* __restrict__ T,
                                      const float* __restrict__ Jeff, const float* __restrict__ aloc,
                                      int lam_begin, int lam_count, long long ncell,
                                      double* __restrict__ out) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    double Jb[kMaxLines], Lc[kMaxLines];
    line_integrals_cell(A, c, ncell, T[c], Jeff, aloc, lam_begin, lam_count, Jb, Lc);
    for (int li = 0; li < A.n_lines; ++li) {
        out[(size_t)(2 * li) * ncell + c] = Jb[li];
        out[(size_t)(2 * li + 1) * ncell + c] = Lc[li];
    }
}

// Gamma n = 0 per cell from line integrals summed over every wavelength of every line.
__global__ void stat_eq_integrals_kernel(AtomDev A, const double* __restrict__ T,
                                         const double* __restrict__ ne,
                                         const double* __restrict__ n_atom,
                                         const double* __restrict__ integ, long long ncell,
                                         double* __restrict__ pops,
                                         unsigned long long* __restrict__ dmax_bits) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rel = 0.0;
    if (c < ncell) {
        double Jb[kMaxLines], Lc[kMaxLines];
        for (int li = 0; li < A.n_lines; ++li) {
            Jb[li] = integ[(size_t)(2 * li) * ncell + c];
            Lc[li] = integ[(size_t)(2 * li + 1) * ncell + c];
        }
        rel = solve_cell(A, c, ncell, T[c], ne[c], n_atom[c], Jb, Lc, pops);
    }
    block_max_to(rel, dmax_bits);
}

}  // namespace

struct rc_atom_s {
    int device = 0;
    AtomDev dev{};
    int n_lambda = 0;
    double* d_grid = nullptr;     // dnu, w, then E/k and g of the levels
    // driver workspace
    float* d_ws = nullptr;
    size_t ws_floats = 0;
    unsigned long long* d_dmax = nullptr;
    double* h_dmax = nullptr;     // pinned
};

namespace {

rc_status launch_stat_eq(rc_atom_t a, const double* T, const double* ne, const double* n_atom,
                         const float* J_eff, const float* alo_c, long long ncell, double* pops,
                         cudaStream_t s, const unsigned char* active = nullptr) {
    cudaError_t e = cudaMemsetAsync(a->d_dmax, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return ncuda(e, "rc_stat_eq");
    stat_eq_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(a->dev, T, ne, n_atom, J_eff,
                                                                   alo_c, ncell, pops, a->d_dmax,
                                                                   active);
    if ((e = cudaGetLastError()) != cudaSuccess) return ncuda(e, "rc_stat_eq launch");
    return RC_OK;
}

rc_status read_dmax(rc_atom_t a, cudaStream_t s, double* out) {
    cudaError_t e = cudaMemcpyAsync(a->h_dmax, a->d_dmax, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return ncuda(e, "rc_stat_eq: reading the maximum change");
    *out = *a->h_dmax;
    return RC_OK;
}

}  // namespace

extern "C" {

rc_status rc_atom_create(const rc_atom_desc* d, rc_atom_t* out) {
    rcx::set_last_error("");
    if (!out) return nfail(RC_ERR_ARG, "rc_atom_create: out is NULL");
    *out = nullptr;
    if (!d || !d->E_eV || !d->g || !d->lower || !d->upper || !d->A_ul)
        return nfail(RC_ERR_ARG, "rc_atom_create: NULL description or array");
    if (d->n_levels < 2 || d->n_levels > kMaxLevels)
        return nfail(RC_ERR_ARG, "rc_atom_create: n_levels must be in [2, 8]");
    if (d->n_lines < 1 || d->n_lines > kMaxLines)
        return nfail(RC_ERR_ARG, "rc_atom_create: n_lines must be in [1, 16]");
    if (d->n_per_line < 2 || d->n_per_line > kMaxPerLine)
        return nfail(RC_ERR_ARG, "rc_atom_create: n_per_line must be in [2, 64]");
    if (!(d->x_max > 0) || !(d->T_ref > 0) || !(d->mass_amu > 0))
        return nfail(RC_ERR_ARG, "rc_atom_create: x_max, T_ref and mass_amu must be positive");
    for (int i = 0; i < d->n_levels; ++i)
        if (!(d->g[i] > 0) || (i > 0 && !(d->E_eV[i] > d->E_eV[i - 1])))
            return nfail(RC_ERR_ARG, "rc_atom_create: weights must be positive, energies ascending");
    rc_atom_s* a = new (std::nothrow) rc_atom_s();
    if (!a) return nfail(RC_ERR_OOM, "rc_atom_create: host allocation");
    cudaGetDevice(&a->device);
    AtomDev& A = a->dev;
    A.n_levels = d->n_levels;
    A.n_lines = d->n_lines;
    A.n_per_line = d->n_per_line;
    for (int i = 0; i < d->n_levels; ++i) {
        A.E_k[i] = d->E_eV[i] * kEV / kK;
        A.g[i] = d->g[i];
    }
    const double m = d->mass_amu * kAmu;
    const double beta = kH * kH / (std::pow(2.0 * kPi * kMe, 1.5) * std::sqrt(kK));
    std::vector<double> grid(2 * (size_t)d->n_lines * d->n_per_line + 2 * kMaxLevels, 0.0);
    double* hdnu = grid.data();
    double* hw = grid.data() + (size_t)d->n_lines * d->n_per_line;
    for (int li = 0; li < d->n_lines; ++li) {
        const int lo = d->lower[li], up = d->upper[li];
        if (lo < 0 || up >= d->n_levels || !(lo < up) || !(d->A_ul[li] > 0)) {
            delete a;
            return nfail(RC_ERR_ARG, "rc_atom_create: bad line levels or A_ul");
        }
        LineConst& L = A.line[li];
        const double dE = (d->E_eV[up] - d->E_eV[lo]) * kEV;
        const double nu0 = dE / kH;
        L.lo = lo;
        L.up = up;
        L.lam0 = li * d->n_per_line;
        L.A = d->A_ul[li];
        L.Bul = L.A * kC * kC / (2.0 * kH * nu0 * nu0 * nu0);
        L.Blu = d->g[up] / d->g[lo] * L.Bul;
        L.hnu_4pi = kH * nu0 / (4.0 * kPi);
        L.dop = nu0 / kC * std::sqrt(2.0 * kK / m);
        const double f_lu = L.A * kEps0 * kMe * kC * kC * kC * d->g[up] /
                            (2.0 * kPi * kQe * kQe * nu0 * nu0 * d->g[lo]);
        // C_lu = n_e beta Omega_lu / (g_l sqrt T) e^-y,  Omega_lu = (8 pi/sqrt 3)(E_Ryd/dE) g_l f_lu P(y)
        L.coll = beta * (8.0 * kPi / std::sqrt(3.0)) * (kRydbergE / dE) * f_lu;
        L.y_T = dE / kK;
        L.glo_gup = d->g[lo] / d->g[up];
        const double dref = nu0 / kC * std::sqrt(2.0 * kK * d->T_ref / m);
        const double step = 2.0 * d->x_max / (double)(d->n_per_line - 1) * dref;
        L.ddnu = step;
        for (int k = 0; k < d->n_per_line; ++k) {
            hdnu[(size_t)li * d->n_per_line + k] = (-d->x_max + 2.0 * d->x_max * k / (d->n_per_line - 1)) * dref;
            hw[(size_t)li * d->n_per_line + k] = (k == 0 || k == d->n_per_line - 1) ? 0.5 * step : step;
        }
    }
    double* hlev = grid.data() + 2 * (size_t)d->n_lines * d->n_per_line;
    for (int i = 0; i < d->n_levels; ++i) {
        hlev[i] = A.E_k[i];
        hlev[kMaxLevels + i] = A.g[i];
    }
    cudaError_t e = cudaMalloc(&a->d_grid, grid.size() * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMemcpy(a->d_grid, grid.data(), grid.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&a->d_dmax, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&a->h_dmax, sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(a->d_grid);
        cudaFree(a->d_dmax);
        delete a;
        return ncuda(e, "rc_atom_create: device tables");
    }
    A.dnu = a->d_grid;
    A.w = a->d_grid + (size_t)d->n_lines * d->n_per_line;
    a->n_lambda = d->n_lines * d->n_per_line;
    *out = a;
    return RC_OK;
}

void rc_atom_destroy(rc_atom_t a) {
    if (!a) return;
    cudaDeviceSynchronize();
    cudaFree(a->d_grid);
    cudaFree(a->d_dmax);
    cudaFree(a->d_ws);
    cudaFreeHost(a->h_dmax);
    delete a;
}

int rc_atom_n_lambda(rc_atom_t a) { return a ? a->n_lambda : 0; }

}  // extern "C"

rc_status rcx::atom_levels(rc_atom_t a, const double** Ek, const double** g, int* nlev,
                           int* n_per_line, int* n_lines) {
    if (!a) return nfail(RC_ERR_ARG, "atom is NULL");
    const double* lev = a->d_grid + 2 * (size_t)a->dev.n_lines * a->dev.n_per_line;
    *Ek = lev;
    *g = lev + kMaxLevels;
    *nlev = a->dev.n_levels;
    *n_per_line = a->dev.n_per_line;
    *n_lines = a->dev.n_lines;
    return RC_OK;
}

extern "C" {

rc_status rc_lte(rc_atom_t a, const double* T, const double* nH, long long ncell, double* ne,
                 double* n_atom, double* pops, void* stream) {
    rcx::set_last_error("");
    if (!a || !T || !nH || !ne || !n_atom || !pops || ncell < 0)
        return nfail(RC_ERR_ARG, "rc_lte: NULL argument or negative ncell");
    if (ncell == 0) return RC_OK;
    const double saha_c = std::pow(2.0 * kPi * kMe * kK / (kH * kH), 1.5);
    lte_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        a->dev, T, nH, ncell, saha_c, kChiH / kK, ne, n_atom, pops);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : ncuda(e, "rc_lte launch");
}

rc_status rc_emis_opac(rc_atom_t a, const double* T, const double* pops, long long ncell,
                       float* chi, float* eta, void* stream) {
    rcx::set_last_error("");
    if (!a || !T || !pops || !chi || !eta || ncell < 0)
        return nfail(RC_ERR_ARG, "rc_emis_opac: NULL argument or negative ncell");
    if (ncell == 0) return RC_OK;
    emis_opac_kernel<<<(unsigned)((ncell + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        a->dev, T, pops, ncell, chi, eta);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : ncuda(e, "rc_emis_opac launch");
}

rc_status rc_stat_eq(rc_atom_t a, const double* T, const double* ne, const double* n_atom,
                     const float* J_eff, const float* alo_c, long long ncell, double* pops,
                     double* max_rel_change, void* stream) {
    rcx::set_last_error("");
    if (!a || !T || !ne || !n_atom || !J_eff || !pops || ncell < 0)
        return nfail(RC_ERR_ARG, "rc_stat_eq: NULL argument or negative ncell");
    if (ncell == 0) {
        if (max_rel_change) *max_rel_change = 0.0;
        return RC_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc_status st = launch_stat_eq(a, T, ne, n_atom, J_eff, alo_c, ncell, pops, s);
    if (st != RC_OK || !max_rel_change) return st;
    return read_dmax(a, s, max_rel_change);
}

rc_status rc_line_integrals(rc_atom_t a, const double* T, const float* J_eff, const float* alo_c,
                            int lambda_begin, int lambda_count, long long ncell, double* out,
                            void* stream) {
    rcx::set_last_error("");
    if (!a || !T || !J_eff || !out || ncell < 0 || lambda_begin < 0 || lambda_count < 0 ||
        lambda_begin + lambda_count > a->n_lambda)
        return nfail(RC_ERR_ARG, "rc_line_integrals: NULL argument or wavelength range outside "
                                 "the atom's grid");
    if (ncell == 0) return RC_OK;
    line_integrals_kernel<<<(unsigned)((ncell + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        a->dev, T, J_eff, alo_c, lambda_begin, lambda_count, ncell, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RC_OK : ncuda(e, "rc_line_integrals launch");
}

rc_status rc_stat_eq_integrals(rc_atom_t a, const double* T, const double* ne,
                               const double* n_atom, const double* integrals, long long ncell,
                               double* pops, double* max_rel_change, void* stream) {
    rcx::set_last_error("");
    if (!a || !T || !ne || !n_atom || !integrals || !pops || ncell < 0)
        return nfail(RC_ERR_ARG, "rc_stat_eq_integrals: NULL argument or negative ncell");
    if (ncell == 0) {
        if (max_rel_change) *max_rel_change = 0.0;
        return RC_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(a->d_dmax, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return ncuda(e, "rc_stat_eq_integrals");
    stat_eq_integrals_kernel<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(
        a->dev, T, ne, n_atom, integrals, ncell, pops, a->d_dmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return ncuda(e, "rc_stat_eq_integrals launch");
    if (!max_rel_change) return RC_OK;
    return read_dmax(a, s, max_rel_change);
}

rc_status rc_nlte_solve(rc_plan_t plan, rc_atom_t a, const double* T, const double* ne,
                        const double* n_atom, double* pops, double tol, int max_iter,
                        int* iterations, double* final_change, double* history, void* stream) {
    rcx::set_last_error("");
    if (!plan || !a || !T || !ne || !n_atom || !pops || max_iter < 1 || !(tol > 0))
        return nfail(RC_ERR_ARG, "rc_nlte_solve: NULL argument, max_iter < 1 or tol <= 0");
    const long long ncell = (long long)plan->nx * plan->nz;
    const int nl = a->n_lambda;
    const size_t need = (size_t)5 * nl * ncell;   // chi, eta, J, J_eff, alo_c
    if (a->ws_floats < need) {
        cudaDeviceSynchronize();
        cudaFree(a->d_ws);
        a->d_ws = nullptr;
        a->ws_floats = 0;
        if (cudaMalloc(&a->d_ws, need * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return nfail(RC_ERR_OOM, "rc_nlte_solve: workspace allocation");
        }
        a->ws_floats = need;
    }
    float* chi = a->d_ws;
    float* eta = chi + (size_t)nl * ncell;
    float* J = eta + (size_t)nl * ncell;
    float* Jeff = J + (size_t)nl * ncell;
    float* aloc = Jeff + (size_t)nl * ncell;
    cudaStream_t s = (cudaStream_t)stream;
    double change = INFINITY;
    int it = 0;
    for (; it < max_iter; ++it) {
        rc_status st = rc_emis_opac(a, T, pops, ncell, chi, eta, stream);
        if (st != RC_OK) return st;
        st = rc_formal_solve_mali(plan, chi, eta, nl, J, nullptr, Jeff, aloc, stream);
        if (st != RC_OK) return st;
        st = launch_stat_eq(a, T, ne, n_atom, Jeff, aloc, ncell, pops, s,
                            plan->sparse ? plan->d_active : nullptr);
        if (st != RC_OK) return st;
        st = read_dmax(a, s, &change);
        if (st != RC_OK) return st;
        if (history) history[it] = change;
        if (change < tol) {
            ++it;
            break;
        }
    }
    if (iterations) *iterations = it;
    if (final_change) *final_change = change;
    if (change < tol) return RC_OK;
    return nfail(RC_ERR_NOT_CONVERGED, "rc_nlte_solve: max_iter reached before tol");
}

}  // extern "C"
