// C ABI, host-side set-up and the propagation driver (one GPU, one stream).
//
// Set-up builds, once per handle: the FFT twiddles, the periodic local potential (on the
// device), the projector sphere tables in gather and scatter order, and the coupling
// blocks D_l I + lambda_l L.S (Eq. Vps-soc, L.S form of Sec. 4.4).  L is obtained by
// applying -i r x grad exactly to the real solid-harmonic polynomials and projecting
// back with exact sphere integrals of monomials.
//
// Each step is the ETRS scheme (propagator reading stated in include/tddft.h):
//   series 1: T_k((H[rho(t), t] - c)/Delta) psi(t), accumulated into both
//             psi~ = Exp(-i dt H) psi  and  phi = Exp(-i dt/2 H) psi  (shared T_k)
//   rho~ = rho(psi~), V~ = V[rho~, t+dt]
//   series 2: psi(t+dt) = Exp(-i dt/2 H[rho~, t+dt]) phi, repeated n_sc times with the
//             corrected density, then rho(t+dt), V(t+dt).
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cstdint>
#include <complex>
#include <map>
#include <array>
#include <string>
#include <type_traits>
#include <vector>

#include "impl.cuh"

using namespace tddft;

namespace {

thread_local std::string g_create_error;

using cd = std::complex<double>;

// ------------------------------------------------------------------ real solid harmonics
// S_{l,mu}(x, y, z) = r^l Y^real_{l,mu}, mu = -l..l, as monomial coefficient maps.
using Mono = std::array<int, 3>;
using Poly = std::map<Mono, double>;

std::vector<Poly> solid_harmonics(int l) {
  const double pi = 3.14159265358979323846;
  std::vector<Poly> out;
  if (l == 0) {
    out.push_back({{{0, 0, 0}, 0.5 / std::sqrt(pi)}});
  } else if (l == 1) {
    const double c = std::sqrt(3.0 / (4.0 * pi));
    out.push_back({{{0, 1, 0}, c}});  // y
    out.push_back({{{0, 0, 1}, c}});  // z
    out.push_back({{{1, 0, 0}, c}});  // x
  } else if (l == 2) {
    const double c = 0.5 * std::sqrt(15.0 / pi);
    const double c0 = 0.25 * std::sqrt(5.0 / pi);
    out.push_back({{{1, 1, 0}, c}});                                              // xy
    out.push_back({{{0, 1, 1}, c}});                                              // yz
    out.push_back({{{0, 0, 2}, 2.0 * c0}, {{2, 0, 0}, -c0}, {{0, 2, 0}, -c0}});   // 3z^2 - r^2
    out.push_back({{{1, 0, 1}, c}});                                              // xz
    out.push_back({{{2, 0, 0}, 0.5 * c}, {{0, 2, 0}, -0.5 * c}});                 // x^2 - y^2
  }
  return out;
}

double poly_eval(const Poly& p, double x, double y, double z) {
  double s = 0.0;
  for (auto& kv : p) s += kv.second * std::pow(x, kv.first[0]) * std::pow(y, kv.first[1]) * std::pow(z, kv.first[2]);
  return s;
}

// (r x grad)_alpha applied to a polynomial (real part of i L_alpha ... times -1): returns Q with L = -i Q.
Poly rxgrad(const Poly& p, int alpha) {
  const int b = (alpha + 1) % 3, c = (alpha + 2) % 3;  // (r x grad)_a = x_b d_c - x_c d_b
  Poly q;
  for (auto& kv : p) {
    const Mono& m = kv.first;
    if (m[c] > 0) {  // x_b d_c
      Mono n = m;
      n[c] -= 1;
      n[b] += 1;
      q[n] += kv.second * m[c];
    }
    if (m[b] > 0) {  // - x_c d_b
      Mono n = m;
      n[b] -= 1;
      n[c] += 1;
      q[n] -= kv.second * m[b];
    }
  }
  return q;
}

// Integral of x^a y^b z^c over the unit sphere.
double sphere_monomial(int a, int b, int c) {
  if ((a & 1) || (b & 1) || (c & 1)) return 0.0;
  return 2.0 * std::tgamma(0.5 * (a + 1)) * std::tgamma(0.5 * (b + 1)) * std::tgamma(0.5 * (c + 1)) /
         std::tgamma(0.5 * (a + b + c + 3));
}

double sphere_inner(const Poly& p, const Poly& q) {
  double s = 0.0;
  for (auto& x : p)
    for (auto& y : q)
      s += x.second * y.second * sphere_monomial(x.first[0] + y.first[0], x.first[1] + y.first[1], x.first[2] + y.first[2]);
  return s;
}

// L_alpha[mu][nu] = <S_mu| L_alpha |S_nu> on the sphere (complex, purely imaginary).
std::vector<std::vector<cd>> angular_momentum(int l, int alpha) {
  auto S = solid_harmonics(l);
  const int n = 2 * l + 1;
  std::vector<std::vector<cd>> L(n, std::vector<cd>(n));
  for (int nu = 0; nu < n; ++nu) {
    Poly q = rxgrad(S[nu], alpha);
    for (int mu = 0; mu < n; ++mu) L[mu][nu] = cd(0.0, -sphere_inner(S[mu], q));
  }
  return L;
}

// ------------------------------------------------------------------ Bessel J_k (Miller)
std::vector<double> bessel_j(int kmax, double z) {
  std::vector<double> J(kmax + 1, 0.0);
  if (z == 0.0) {
    J[0] = 1.0;
    return J;
  }
  const double az = std::fabs(z);
  const int start = std::max(kmax, (int)az) + 60 + (int)(2.0 * std::sqrt(az + 1.0) * 10.0);
  std::vector<double> w(start + 2, 0.0);
  w[start + 1] = 0.0;
  w[start] = 1e-300;
  for (int k = start; k >= 1; --k) {
    w[k - 1] = 2.0 * k / az * w[k] - w[k + 1];
    if (std::fabs(w[k - 1]) > 1e250) {
      for (int j = k - 1; j <= start + 1; ++j) w[j] *= 1e-250;
    }
  }
  double norm = w[0];
  for (int k = 2; k <= start; k += 2) norm += 2.0 * w[k];
  for (int k = 0; k <= kmax; ++k) {
    double v = w[k] / norm;
    if (z < 0.0 && (k & 1)) v = -v;
    J[k] = v;
  }
  return J;
}

int chebyshev_order(double z, double tol) {
  const int kmax = (int)std::fabs(z) + 400;
  auto J = bessel_j(kmax, z);
  for (int k = (int)std::floor(std::fabs(z)) + 1; k <= kmax; ++k)
    if (std::fabs(J[k]) < tol) return k - 1;
  return kmax;
}

}  // namespace

namespace tddft {
// Message for failures that have no handle (tddft_create, tddft_hartree_noalloc).
void set_global_error(const std::string& msg) { g_create_error = msg; }
}  // namespace tddft

// =================================================================== context

struct tddft_ctx {
  // configuration
  int prec = 0, proj_mode = 0, N = 0;
  size_t N3 = 0;
  double L[3] = {0, 0, 0}, omega = 0, dV = 0;
  int natoms = 0, lmax = 0, nlm = 0;
  std::vector<double> pos, Zat, rcat;
  double r_cut = 0;
  int nk = 0, nb = 0, nkb = 0;
  std::vector<double> kpts, kw, occ, wf;
  double dt = 0;
  int exp_kind = 0, exp_order = 0, n_sc = 0, xc = 1, spin_mode = 0;
  double cheb_tol = 0, sc_tol = 0, emin_user = 0, emax_user = 0;
  std::vector<double> ft, fA, fB;
  // propagation state
  bool have_states = false;
  double t = 0, emin = 0, emax = 0, nl_bound = 0, kin_max = 0;
  int K_full = 0, K_half = 0;
  std::vector<cd> cf_full, cf_half;
  bool use_tma = false;      // FP32 xy passes fed by bulk asynchronous copies
  bool epi_pairs = false;    // epilogue threads take one point of two spinors
  bool epi_fuse = false;     // tensor-core projectors: scatter and Chebyshev epilogue in one kernel
  // device memory
  cudaStream_t st = nullptr;
  // second stream for the projector gather, which runs beside the FFT passes of the same term
  // (it only reads T_k; fork and join events order it after the previous epilogue and before
  // the next one)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<void*> allocs;
  void *psi = nullptr, *phi = nullptr, *pred = nullptr, *Ta = nullptr, *Tb = nullptr, *tmp = nullptr;
  void *cbuf = nullptr, *dcbuf = nullptr, *tw = nullptr;
  double2 *tw64 = nullptr, *hart = nullptr, *stage = nullptr;
  size_t stage_elems = 0;
  double* rho_part = nullptr;  // band-group partial densities
  double *rho = nullptr, *rho2 = nullptr, *rho3 = nullptr, *V = nullptr, *Vnew = nullptr, *vloc = nullptr,
         *vH = nullptr, *exc = nullptr, *vxc4 = nullptr, *wf_d = nullptr, *red = nullptr, *Bd = nullptr;
  float *Vf = nullptr, *Vnewf = nullptr;
  int* flag = nullptr;
  // projector tables (typed views over the raw allocations)
  int *g_ptr = nullptr, *g_idx = nullptr, *s_ptr = nullptr, *s_atom = nullptr;
  size_t n_entries = 0;
  double2* Tsoc = nullptr;   // [natoms][3][2 nlm][2 nlm] 2 i [D_a, S_i] (spin-orbit torque)
  double* tq = nullptr;       // torque partial sums: [nkb][3] spin-orbit, then 6 field sums
  double* red_part = nullptr;  // partials of the two-pass reductions (band dots, field sums)
  int* owner = nullptr;      // nearest atom of each grid point (per-atom moments)
  double* atom_sums = nullptr;
  // tile-centric tensor-core projectors (proj_mode TF32, TF32X3, BF16X3, F16X3)
  bool tile = false;
  TileDev td;
  float* tile_part = nullptr;  // gather partial products, nk * groups * td.part_layer floats
  void* vnl = nullptr;         // V_NL T_k from the tensor-core scatter (spinor layout)
  int* tc_err = nullptr;     // wait errors: bit 1 tensor-core projector, bit 2 bulk-copy FFT pass
  void *g_tab = nullptr, *s_tab = nullptr, *Dmat = nullptr;
  void *g_row = nullptr, *s_row = nullptr, *nrm = nullptr;
  // bookkeeping
  std::string err;
  long long launches = 0;
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[kNumCls];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  double alg_bytes[kNumCls] = {0, 0, 0, 0, 0, 0, 0, 0};  // algorithmic DRAM bytes while profiling

  size_t psi_elems() const { return (size_t)nkb * 2 * N3; }
  size_t rsize() const { return prec == TDDFT_FP64 ? sizeof(double) : sizeof(float); }

  template <typename R> ProjTables<R> tables() const {
    ProjTables<R> p;
    p.natoms = natoms;
    p.nlm = nlm;
    p.ntab = 3 + nlm;
    p.g_ptr = g_ptr;
    p.g_idx = g_idx;
    p.g_tab = (const R*)g_tab;
    p.s_ptr = s_ptr;
    p.s_atom = s_atom;
    p.s_tab = (const R*)s_tab;
    p.Dmat = (const R*)Dmat;
    p.g_row = (const R*)g_row;
    p.s_row = (const R*)s_row;
    p.nrm = (const R*)nrm;
    const double pi = 3.14159265358979323846;  // the constants of solid_harmonics()
    p.yc[0] = (R)(0.5 / std::sqrt(pi));
    p.yc[1] = (R)std::sqrt(3.0 / (4.0 * pi));
    p.yc[2] = (R)(0.5 * std::sqrt(15.0 / pi));
    p.yc[3] = (R)(0.25 * std::sqrt(5.0 / pi));
    return p;
  }

  tddft_status fail(tddft_status s, const std::string& m) {
    err = m;
    return s;
  }
  tddft_status cuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TDDFT_OK;
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TDDFT_ERR_OOM : TDDFT_ERR_CUDA;
  }
  template <typename T> tddft_status alloc(T** p, size_t bytes, const char* what) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      err = std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e);
      return TDDFT_ERR_OOM;
    }
    allocs.push_back(q);
    *p = (T*)q;
    return TDDFT_OK;
  }
  // Launch wrapper: counts launches and records CUDA events around them when profiling.
  template <class F> tddft_status launch(int cls, const char* what, F&& f, double bytes = 0.0) {
    return launch_on(st, cls, what, f, bytes);
  }
  template <class F> tddft_status launch_on(cudaStream_t s, int cls, const char* what, F&& f, double bytes = 0.0) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (prof) {
      if (ev_used == ev_pool.size()) {
        cudaEvent_t x, y;
        cudaEventCreate(&x);
        cudaEventCreate(&y);
        ev_pool.push_back({x, y});
      }
      a = ev_pool[ev_used].first;
      b = ev_pool[ev_used].second;
      ++ev_used;
      cudaEventRecord(a, s);
    }
    cudaError_t e = f();
    if (prof) {
      cudaEventRecord(b, s);
      ev[cls].push_back({a, b});
      alg_bytes[cls] += bytes;
    }
    ++launches;
    return cuda(e, what);
  }
  void field_at(double tt, double A[3], double B[3]) const {
    for (int a = 0; a < 3; ++a) A[a] = B[a] = 0.0;
    const int nt = (int)ft.size();
    if (nt == 0) return;
    if (tt <= ft[0] || nt == 1) {
      for (int a = 0; a < 3; ++a) { A[a] = fA[a]; B[a] = fB[a]; }
      return;
    }
    if (tt >= ft[nt - 1]) {
      for (int a = 0; a < 3; ++a) { A[a] = fA[3 * (nt - 1) + a]; B[a] = fB[3 * (nt - 1) + a]; }
      return;
    }
    const int j = (int)(std::upper_bound(ft.begin(), ft.end(), tt) - ft.begin());
    const double t0 = ft[j - 1], t1 = ft[j];
    const double w = (tt - t0) / (t1 - t0);
    for (int a = 0; a < 3; ++a) {
      A[a] = (1.0 - w) * fA[3 * (j - 1) + a] + w * fA[3 * j + a];
      B[a] = (1.0 - w) * fB[3 * (j - 1) + a] + w * fB[3 * j + a];
    }
  }
  // A(t) and the external field seen by the spin: all of B (non-collinear), its component along
  // the quantisation axis z (collinear), none (unpolarised).
  void fields(double tt, double A[3], double B[3]) const {
    field_at(tt, A, B);
    if (spin_mode == TDDFT_SPIN_COLLINEAR) B[0] = B[1] = 0.0;
    if (spin_mode == TDDFT_SPIN_UNPOLARISED) B[0] = B[1] = B[2] = 0.0;
  }
  double kinetic_max_for(const double s[3]) const {
    const double pi = 3.14159265358979323846;
    double tot = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double g = 2.0 * pi / L[a];
      const double lo = g * (-(N / 2)) + s[a], hi = g * (N / 2 - 1) + s[a];
      tot += std::max(lo * lo, hi * hi);
    }
    return 0.5 * tot;
  }
};

namespace {

tddft_status free_all(tddft_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  for (auto& e : c->ev_pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  c->ev_pool.clear();
  return TDDFT_OK;
}

bool supported_n(int n) {
  static const int ok[] = {8, 12, 16, 24, 32, 48, 64, 96};
  for (int v : ok)
    if (v == n) return true;
  return false;
}

// ------------------------------------------------------------------ projector tables
struct HostTables {
  std::vector<int> g_ptr, g_idx, s_ptr, s_atom;
  std::vector<double> g_tab, s_tab;  // [entries][3 + nlm]
  std::vector<double> g_row, s_row;  // [entries][4]: d, exp(-|d|^2 / (2 w^2))
  std::vector<double> nrm;           // [natoms][4]: N_0, N_1, N_2, 0
  std::vector<double> Dmat;          // [natoms][2nlm][2nlm][2]
  double nl_bound = 0.0;
};

tddft_status build_tables(tddft_ctx* c, const tddft_projectors* pj, const int* species, HostTables& ht) {
  const int N = c->N, nlm = c->nlm, tab = 3 + nlm;
  const double pi = 3.14159265358979323846;
  std::vector<std::vector<Poly>> S(c->lmax + 1);
  for (int l = 0; l <= c->lmax; ++l) S[l] = solid_harmonics(l);
  ht.g_ptr.assign(c->natoms + 1, 0);
  ht.nrm.assign(4 * (size_t)c->natoms, 0.0);
  std::vector<std::vector<double>> per_atom_row(c->natoms);
  std::vector<std::vector<double>> per_atom_tab(c->natoms);
  std::vector<std::vector<int>> per_atom_idx(c->natoms);
  const double h[3] = {c->L[0] / N, c->L[1] / N, c->L[2] / N};
  for (int a = 0; a < c->natoms; ++a) {
    const int s = species[a];
    const double w = pj->width[s];
    double Nl[3];
    for (int l = 0; l <= c->lmax; ++l) Nl[l] = std::sqrt(2.0 / (std::tgamma(l + 1.5) * std::pow(w, 2 * l + 3)));
    for (int l = 0; l <= c->lmax; ++l) ht.nrm[4 * (size_t)a + l] = Nl[l];
    const double* R = &c->pos[3 * a];
    std::vector<double> dz(N), dy(N), dx(N);
    for (int i = 0; i < N; ++i) {
      double v;
      v = i * h[0] - R[0]; dx[i] = v - c->L[0] * std::nearbyint(v / c->L[0]);
      v = i * h[1] - R[1]; dy[i] = v - c->L[1] * std::nearbyint(v / c->L[1]);
      v = i * h[2] - R[2]; dz[i] = v - c->L[2] * std::nearbyint(v / c->L[2]);
    }
    // the cut |d| < r_cut is applied with a 1e-10 relative margin so that points lying on the
    // sphere in exact arithmetic are excluded whatever the rounding of |d|^2
    const double rc2 = c->r_cut * c->r_cut * (1.0 - 1e-10);
    for (int z = 0; z < N; ++z) {
      if (dz[z] * dz[z] >= rc2) continue;
      for (int y = 0; y < N; ++y) {
        if (dz[z] * dz[z] + dy[y] * dy[y] >= rc2) continue;
        for (int x = 0; x < N; ++x) {
          const double r2 = dx[x] * dx[x] + dy[y] * dy[y] + dz[z] * dz[z];
          if (!(r2 < rc2)) continue;
          per_atom_idx[a].push_back((z * N + y) * N + x);
          per_atom_tab[a].push_back(dx[x]);
          per_atom_tab[a].push_back(dy[y]);
          per_atom_tab[a].push_back(dz[z]);
          const double g = std::exp(-r2 / (2.0 * w * w));
          per_atom_row[a].insert(per_atom_row[a].end(), {dx[x], dy[y], dz[z], g});
          for (int l = 0; l <= c->lmax; ++l)
            for (int mu = 0; mu < 2 * l + 1; ++mu)
              per_atom_tab[a].push_back(Nl[l] * g * poly_eval(S[l][mu], dx[x], dy[y], dz[z]));
        }
      }
    }
    ht.g_ptr[a + 1] = ht.g_ptr[a] + (int)per_atom_idx[a].size();
  }
  for (int a = 0; a < c->natoms; ++a) {
    ht.g_idx.insert(ht.g_idx.end(), per_atom_idx[a].begin(), per_atom_idx[a].end());
    ht.g_tab.insert(ht.g_tab.end(), per_atom_tab[a].begin(), per_atom_tab[a].end());
    ht.g_row.insert(ht.g_row.end(), per_atom_row[a].begin(), per_atom_row[a].end());
  }
  // scatter order: counting sort by grid point, atoms ascending
  const size_t N3 = c->N3;
  const size_t ne = ht.g_idx.size();
  ht.s_ptr.assign(N3 + 1, 0);
  for (size_t e = 0; e < ne; ++e) ht.s_ptr[ht.g_idx[e] + 1]++;
  for (size_t i = 0; i < N3; ++i) ht.s_ptr[i + 1] += ht.s_ptr[i];
  ht.s_atom.assign(ne, 0);
  ht.s_tab.assign(ne * tab, 0.0);
  ht.s_row.assign(ne * 4, 0.0);
  std::vector<int> fill(ht.s_ptr.begin(), ht.s_ptr.end() - 1);
  for (int a = 0; a < c->natoms; ++a)
    for (int e = ht.g_ptr[a]; e < ht.g_ptr[a + 1]; ++e) {
      const int dst = fill[ht.g_idx[e]]++;
      ht.s_atom[dst] = a;
      std::memcpy(&ht.s_tab[(size_t)dst * tab], &ht.g_tab[(size_t)e * tab], sizeof(double) * tab);
      std::memcpy(&ht.s_row[(size_t)dst * 4], &ht.g_row[(size_t)e * 4], sizeof(double) * 4);
    }
  // coupling blocks D_l I + lambda_l L.S on (p = l^2 + mu + l, sigma), index 2 p + sigma
  const int M = 2 * nlm;
  ht.Dmat.assign((size_t)c->natoms * M * M * 2, 0.0);
  const cd sig[3][2][2] = {{{0.0, 1.0}, {1.0, 0.0}},
                           {{0.0, cd(0.0, -1.0)}, {cd(0.0, 1.0), 0.0}},
                           {{1.0, 0.0}, {0.0, -1.0}}};
  std::vector<std::vector<std::vector<cd>>> Lm[3];
  for (int al = 0; al < 3; ++al)
    for (int l = 0; l <= c->lmax; ++l) Lm[al].push_back(angular_momentum(l, al));
  // ||V_NL|| = ||P D P^dagger|| <= max_a ||D_a|| ||P^dagger P||; ||P^dagger P|| is bounded by the
  // largest Gershgorin row sum of the Gram matrix of all projectors: exact overlaps within an
  // atom (the phases cancel), sum_r |beta_ap| |beta_bq| dV between atoms.
  std::vector<double> Sabs(c->N3, 0.0);  // sum over all entries at r of |beta|
  for (int a = 0; a < c->natoms; ++a)
    for (int e = ht.g_ptr[a]; e < ht.g_ptr[a + 1]; ++e) {
      const double* t = &ht.g_tab[(size_t)e * tab + 3];
      for (int p = 0; p < nlm; ++p) Sabs[ht.g_idx[e]] += std::fabs(t[p]);
    }
  double dmax_all = 0.0, gmax_all = 0.0;
  for (int a = 0; a < c->natoms; ++a) {
    const int s = species[a];
    double* Da = &ht.Dmat[(size_t)a * M * M * 2];
    double dmax = 0.0;
    for (int l = 0; l <= c->lmax; ++l) {
      const double Dl = pj->D[s * (c->lmax + 1) + l], lam = pj->lambda_so[s * (c->lmax + 1) + l];
      dmax = std::max(dmax, std::fabs(Dl + lam * 0.5 * l));
      if (l > 0) dmax = std::max(dmax, std::fabs(Dl - lam * 0.5 * (l + 1)));
      const int p0 = l * l, nl = 2 * l + 1;
      for (int mu = 0; mu < nl; ++mu)
        for (int nu = 0; nu < nl; ++nu)
          for (int s1 = 0; s1 < 2; ++s1)
            for (int s2 = 0; s2 < 2; ++s2) {
              cd v = (mu == nu && s1 == s2) ? cd(Dl, 0.0) : cd(0.0, 0.0);
              for (int al = 0; al < 3; ++al) v += lam * Lm[al][l][mu][nu] * 0.5 * sig[al][s1][s2];
              const int row = 2 * (p0 + mu) + s1, col = 2 * (p0 + nu) + s2;
              Da[(row * M + col) * 2] = v.real();
              Da[(row * M + col) * 2 + 1] = v.imag();
            }
    }
    // Gershgorin row sums of this atom's rows of the full Gram matrix
    std::vector<double> G((size_t)nlm * nlm, 0.0), inter(nlm, 0.0);
    for (int e = ht.g_ptr[a]; e < ht.g_ptr[a + 1]; ++e) {
      const double* t = &ht.g_tab[(size_t)e * tab + 3];
      double own = 0.0;
      for (int q = 0; q < nlm; ++q) own += std::fabs(t[q]);
      const double other = Sabs[ht.g_idx[e]] - own;
      for (int p = 0; p < nlm; ++p) {
        for (int q = 0; q < nlm; ++q) G[p * nlm + q] += t[p] * t[q] * c->dV;
        inter[p] += std::fabs(t[p]) * other * c->dV;
      }
    }
    for (int p = 0; p < nlm; ++p) {
      double rs = inter[p];
      for (int q = 0; q < nlm; ++q) rs += std::fabs(G[p * nlm + q]);
      gmax_all = std::max(gmax_all, rs);
    }
    dmax_all = std::max(dmax_all, dmax);
  }
  const double bound = dmax_all * gmax_all;
  ht.nl_bound = bound;
  (void)pi;
  return TDDFT_OK;
}

// ------------------------------------------------------------------ brick tables of the tensor-core projectors
// Rounding of the operand values to the tensor-core element kinds (round to nearest; TF32 ties
// away from zero, as the hardware conversion does; BF16 and FP16 ties to even).
uint32_t f32_bits(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
}
float bits_f32(uint32_t u) {
  float x;
  std::memcpy(&x, &u, 4);
  return x;
}
uint32_t to_tf32(float x) { return (f32_bits(x) + 0x1000u) & 0xFFFFE000u; }
uint32_t to_bf16(float x) {
  const uint32_t u = f32_bits(x);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}
uint32_t to_f16(float f) {
  const uint32_t x = f32_bits(f);
  const uint32_t sign = (x >> 16) & 0x8000u;
  const int e = (int)((x >> 23) & 0xFFu) - 127 + 15;
  uint32_t m = x & 0x7FFFFFu;
  if (((x >> 23) & 0xFFu) == 0xFFu) return sign | 0x7C00u | (m ? 0x200u : 0u);
  if (e >= 31) return sign | 0x7C00u;
  if (e <= 0) {  // subnormal half: value = hm 2^-24
    if (e < -10) return sign;
    m |= 0x800000u;
    const int shift = 14 - e;
    uint32_t hm = m >> shift;
    const uint32_t rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1);
    if (rem > half || (rem == half && (hm & 1u))) ++hm;
    return sign | hm;
  }
  uint32_t r = sign | ((uint32_t)e << 10) | (m >> 13);
  const uint32_t rem = m & 0x1FFFu;
  if (rem > 0x1000u || (rem == 0x1000u && (r & 1u))) ++r;  // a carry rounds into the exponent
  return r;
}
double from_kind(int ek, uint32_t v) {
  if (ek == TILE_TF32) return bits_f32(v);
  if (ek == TILE_BF16) return bits_f32(v << 16);
  const uint32_t sign = (v & 0x8000u) << 16, e = (v >> 10) & 0x1Fu, m = v & 0x3FFu;
  if (e == 0) return (sign ? -1.0 : 1.0) * std::ldexp((double)m, -24);
  if (e == 31) return bits_f32(sign | 0x7F800000u | (m << 13));
  return bits_f32(sign | ((e - 15 + 127) << 23) | (m << 13));
}
uint32_t to_kind(int ek, double x) {
  if (ek == TILE_TF32) return to_tf32((float)x);
  if (ek == TILE_BF16) return to_bf16((float)x);
  return to_f16((float)x);
}

struct TileHost {
  int BX = 32, nbx = 0, nby = 0, nbz = 0, smax = 0, kch_max = 0;
  std::vector<int> it_brick, it_nslot, it_npad, it_kch, slot_atom, a_ptr, a_item, a_slot;
  std::vector<long long> it_goff, it_soff, it_poff;
  std::vector<float> slot_delta;          // [nitems][smax][4]
  std::vector<unsigned char> g_tab, s_tab;
  long long part_layer = 0;
};

// Bricks of BX x 8 x 8 points; per brick the atom images ("slots") whose spheres reach into it,
// and the real projector values beta_{slot,p}(r) of every brick point (from the per-atom entries
// of build_tables, FP64), rounded to the operand kind in the swizzled K-major layout:
//   gather  (operand B): per chunk of 128-byte rows of points, npad rows (slot, p) x 128 bytes;
//   scatter (operand A): per tile of 128 points and chunk of 128-byte rows of (slot, p), 128 rows.
// With three products each chunk holds the hi part, then lo = value - hi.
tddft_status build_tile_tables(tddft_ctx* c, const HostTables& ht, int ek, int terms, TileHost& th) {
  const int N = c->N, nlm = c->nlm;
  if (N % 16 != 0) return c->fail(TDDFT_ERR_UNSUPPORTED, "tensor-core projectors need a grid size divisible by 16");
  th.BX = (N % 32 == 0) ? 32 : 16;
  th.nbx = N / th.BX;
  th.nby = th.nbz = N / 8;
  th.smax = 256 / nlm;
  const int esz = (ek == TILE_TF32) ? 4 : 2, epr = 128 / esz, npart = (terms == 3) ? 2 : 1;
  const int pts = th.BX * 64, nch = pts / epr, ntile = pts / 128;
  const int nbr = th.nbx * th.nby * th.nbz;
  const int tab = 3 + nlm;
  const double h[3] = {c->L[0] / N, c->L[1] / N, c->L[2] / N};
  // slot of (atom, image) in each brick, in order of first appearance (atoms ascending)
  std::vector<std::vector<long long>> keys(nbr);
  struct Ent { int brick, slot, local; size_t e; };
  std::vector<Ent> ents;
  ents.reserve(ht.g_idx.size());
  for (int a = 0; a < c->natoms; ++a) {
    for (int e = ht.g_ptr[a]; e < ht.g_ptr[a + 1]; ++e) {
      const int idx = ht.g_idx[e];
      const int x = idx % N, y = (idx / N) % N, z = idx / (N * N);
      const double* d = &ht.g_tab[(size_t)e * tab];
      int img[3];
      const int xyz[3] = {x, y, z};
      for (int ax = 0; ax < 3; ++ax)
        img[ax] = (int)std::lround((xyz[ax] * h[ax] - d[ax] - c->pos[3 * a + ax]) / c->L[ax]);
      const long long key = (long long)a * 27 + (img[0] + 1) * 9 + (img[1] + 1) * 3 + (img[2] + 1);
      const int b = (x / th.BX) + th.nbx * ((y / 8) + th.nby * (z / 8));
      auto& kv = keys[b];
      int sl = -1;
      for (int i = 0; i < (int)kv.size(); ++i)
        if (kv[i] == key) { sl = i; break; }
      if (sl < 0) {
        sl = (int)kv.size();
        kv.push_back(key);
      }
      const int local = (x % th.BX) + th.BX * ((y % 8) + 8 * (z % 8));
      ents.push_back({b, sl, local, (size_t)e});
    }
  }
  // every brick is an item (the fused epilogue visits every point); bricks no sphere reaches have
  // no slots, and the gather and the plain scatter skip them
  std::vector<int> item_of(nbr, -1);
  for (int b = 0; b < nbr; ++b) {
    if ((int)keys[b].size() > th.smax)
      return c->fail(TDDFT_ERR_UNSUPPORTED, "too many projector spheres reach one brick for the tensor-core path");
    item_of[b] = (int)th.it_brick.size();
    th.it_brick.push_back(b);
  }
  const int nit = (int)th.it_brick.size();
  th.it_nslot.resize(nit);
  th.it_npad.resize(nit);
  th.it_kch.resize(nit);
  th.it_goff.resize(nit);
  th.it_soff.resize(nit);
  th.it_poff.resize(nit);
  th.slot_atom.assign((size_t)nit * th.smax, 0);
  th.slot_delta.assign((size_t)nit * th.smax * 4, 0.0f);
  long long goff = 0, soff = 0, poff = 0;
  for (int i = 0; i < nit; ++i) {
    const int b = th.it_brick[i];
    const int ns = (int)keys[b].size();
    th.it_nslot[i] = ns;
    th.it_npad[i] = ns ? std::max(16, (ns * nlm + 15) / 16 * 16) : 0;
    th.it_kch[i] = (ns * nlm + epr - 1) / epr;
    th.kch_max = std::max(th.kch_max, th.it_kch[i]);
    th.it_goff[i] = goff;
    th.it_soff[i] = soff;
    th.it_poff[i] = poff;
    goff += (long long)nch * npart * th.it_npad[i] * 128;
    soff += (long long)ntile * th.it_kch[i] * npart * 128 * 128;
    poff += (long long)ns * nlm * 128;
    const int bx = b % th.nbx, by = (b / th.nbx) % th.nby, bz = b / (th.nbx * th.nby);
    const double rb[3] = {bx * th.BX * h[0], by * 8 * h[1], bz * 8 * h[2]};
    for (int sl = 0; sl < ns; ++sl) {
      const long long key = keys[b][sl];
      const int a = (int)(key / 27), r = (int)(key % 27);
      const int img[3] = {r / 9 - 1, (r / 3) % 3 - 1, r % 3 - 1};
      th.slot_atom[(size_t)i * th.smax + sl] = a;
      for (int ax = 0; ax < 3; ++ax)
        th.slot_delta[((size_t)i * th.smax + sl) * 4 + ax] =
            (float)(rb[ax] - (c->pos[3 * a + ax] + img[ax] * c->L[ax]));
    }
  }
  th.part_layer = poff;
  // dense projector values per item: vals[item][slot * nlm + p][local point]
  std::vector<long long> vbase(nit + 1, 0);
  for (int i = 0; i < nit; ++i) vbase[i + 1] = vbase[i] + (long long)th.it_nslot[i] * nlm * pts;
  std::vector<double> vals((size_t)vbase[nit], 0.0);
  for (const Ent& en : ents) {
    const int i = item_of[en.brick];
    const double* t = &ht.g_tab[en.e * tab + 3];
    for (int p = 0; p < nlm; ++p) vals[(size_t)vbase[i] + ((size_t)en.slot * nlm + p) * pts + en.local] = t[p];
  }
  auto sw = [](size_t off) { return off ^ (((off >> 7) & 7u) << 4); };
  auto store = [&](std::vector<unsigned char>& dst, size_t base, size_t off, uint32_t v) {
    unsigned char* q = dst.data() + base + sw(off);
    if (esz == 4) std::memcpy(q, &v, 4);
    else { const uint16_t w = (uint16_t)v; std::memcpy(q, &w, 2); }
  };
  th.g_tab.assign((size_t)goff, 0);
  th.s_tab.assign((size_t)soff, 0);
  for (int i = 0; i < nit; ++i) {
    const int ns = th.it_nslot[i], npad = th.it_npad[i], kch = th.it_kch[i];
    const double* v = &vals[(size_t)vbase[i]];
    for (int n = 0; n < ns * nlm; ++n)
      for (int lp = 0; lp < pts; ++lp) {
        const double x = v[(size_t)n * pts + lp];
        if (x == 0.0) continue;
        const uint32_t hi = to_kind(ek, x);
        const uint32_t lo = to_kind(ek, x - from_kind(ek, hi));
        // gather: chunk lp / epr, row n, element lp % epr
        const int ch = lp / epr, el = lp % epr;
        const size_t gb = (size_t)th.it_goff[i] + (size_t)ch * npart * npad * 128;
        store(th.g_tab, gb, (size_t)n * 128 + (size_t)el * esz, hi);
        if (npart == 2) store(th.g_tab, gb + (size_t)npad * 128, (size_t)n * 128 + (size_t)el * esz, lo);
        // scatter: tile lp / 128, K chunk n / epr, row lp % 128, element n % epr
        const int tl = lp / 128, row = lp % 128, kc = n / epr, ke = n % epr;
        const size_t sb = (size_t)th.it_soff[i] + ((size_t)tl * kch + kc) * npart * 128 * 128;
        store(th.s_tab, sb, (size_t)row * 128 + (size_t)ke * esz, hi);
        if (npart == 2) store(th.s_tab, sb + 128 * 128, (size_t)row * 128 + (size_t)ke * esz, lo);
      }
  }
  // (item, slot) pairs of every atom, items ascending
  th.a_ptr.assign(c->natoms + 1, 0);
  for (int i = 0; i < nit; ++i)
    for (int sl = 0; sl < th.it_nslot[i]; ++sl) th.a_ptr[th.slot_atom[(size_t)i * th.smax + sl] + 1]++;
  for (int a = 0; a < c->natoms; ++a) th.a_ptr[a + 1] += th.a_ptr[a];
  th.a_item.assign(th.a_ptr[c->natoms], 0);
  th.a_slot.assign(th.a_ptr[c->natoms], 0);
  std::vector<int> fill(th.a_ptr.begin(), th.a_ptr.end() - 1);
  for (int i = 0; i < nit; ++i)
    for (int sl = 0; sl < th.it_nslot[i]; ++sl) {
      const int a = th.slot_atom[(size_t)i * th.smax + sl];
      th.a_item[fill[a]] = i;
      th.a_slot[fill[a]] = sl;
      ++fill[a];
    }
  return TDDFT_OK;
}

template <typename R>
tddft_status upload_typed(tddft_ctx* c, void** dst, const std::vector<double>& src, const char* what) {
  std::vector<R> tmp(src.begin(), src.end());
  tddft_status s = c->alloc(dst, tmp.size() * sizeof(R), what);
  if (s) return s;
  return c->cuda(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice), what);
}

template <typename T>
tddft_status upload(tddft_ctx* c, T** dst, const std::vector<T>& src, const char* what) {
  tddft_status s = c->alloc(dst, src.size() * sizeof(T), what);
  if (s) return s;
  return c->cuda(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice), what);
}

// ------------------------------------------------------------------ potential pipeline
tddft_status hartree(tddft_ctx* c, const double* rho) {
  ZParams zp{};
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < 3; ++a) zp.gs[a] = 2.0 * pi / c->L[a];
  zp.scale = 1.0 / (double)c->N3;
  tddft_status s;
  if ((s = c->launch(KC_POT, "density to complex", [&] { return launch_density_to_complex(c->st, c->N3, rho, c->hart); }))) return s;
  if ((s = c->launch(KC_POT, "hartree fft xy", [&] { return launch_fft_xy<double>(c->st, c->N, c->hart, c->hart, 1, c->tw64, false); }))) return s;
  if ((s = c->launch(KC_POT, "hartree fft z", [&] { return launch_fft_z<double>(c->st, c->N, c->hart, 1, c->tw64, Z_POISSON, zp); }))) return s;
  if ((s = c->launch(KC_POT, "hartree ifft xy", [&] { return launch_fft_xy<double>(c->st, c->N, c->hart, c->hart, 1, c->tw64, true); }))) return s;
  return c->launch(KC_POT, "hartree real part", [&] { return launch_complex_real_part(c->st, c->N3, c->hart, c->vH, 1.0); });
}

// rho (4 x N3) -> V (FP64) and, in mixed precision, its FP32 copy.
tddft_status potential(tddft_ctx* c, const double* rho, double tt, double* Vout, float* Vfout) {
  double A[3], B[3];
  c->fields(tt, A, B);
  tddft_status s = hartree(c, rho);
  if (s) return s;
  return c->launch(KC_POT, "potential", [&] {
    return launch_potential(c->st, c->N3, rho, c->vH, c->vloc, B, c->xc, c->spin_mode, Vout, Vfout, c->exc, c->vxc4);
  });
}

template <typename R> tddft_status density(tddft_ctx* c, const void* psi, double* rho) {
  const double by = (double)c->psi_elems() * 2 * sizeof(R) + 4.0 * c->N3 * sizeof(double);
  return c->launch(KC_DENS, "density", [&] {
    return launch_density<R>(c->st, c->N3, psi, c->nkb, c->wf_d, rho, c->rho_part);
  }, by);
}

tddft_status window_check(tddft_ctx* c, const double* V) {
  return c->launch(KC_OTHER, "window check", [&] {
    return launch_check_window(c->st, c->N3, V, c->emin, c->emax, c->kin_max, c->nl_bound, c->flag);
  });
}

template <typename R> const R* vsel(tddft_ctx* c, bool cur) {
  if (c->prec == TDDFT_FP64) return (const R*)(cur ? c->V : c->Vnew);
  return (const R*)(cur ? (void*)c->Vf : (void*)c->Vnewf);
}

void fill_shifts(tddft_ctx* c, const double A[3], double (*shift)[3]) {
  for (int k = 0; k < c->nk; ++k)
    for (int a = 0; a < 3; ++a) shift[k][a] = c->kpts[3 * k + a] + A[a];
}

// One xy pass over nbatch spinor components (FP32: the bulk-copy form where it applies).
template <typename R> cudaError_t xy_pass(tddft_ctx* c, const void* in, void* out, int nbatch, bool inv) {
  if constexpr (std::is_same<R, float>::value)
    if (c->use_tma && fft_xy_tma_supported(c->N))
      return launch_fft_xy_tma(c->st, c->N, in, out, nbatch, c->tw, inv, c->tc_err);
  return launch_fft_xy<R>(c->st, c->N, in, out, nbatch, c->tw, inv);
}

// The pointwise epilogue (one point of two spinors per thread unless switched off).
template <typename R>
cudaError_t epilogue(tddft_ctx* c, const void* kin, const void* Tk, const void* Tkm1, void* Tout, void* acc1,
                     void* acc2, const R* V, const ProjTables<R>& pt, const void* dc, int nkb, const EpiParams& ep) {
  EpiParams e = ep;
  e.spinor_pairs = c->epi_pairs ? 1 : 0;
  // with the tensor-core projectors (tables without atoms) V_NL T_k waits in vnl
  const void* kin2 = (c->tile && pt.natoms == 0) ? c->vnl : nullptr;
  return launch_epilogue<R>(c->st, c->N, kin, kin2, Tk, Tkm1, Tout, acc1, acc2, V, pt, dc, nkb, e);
}

// Kinetic part of H on all spinors: out = T in (three FFT passes).
template <typename R> tddft_status kinetic(tddft_ctx* c, const void* in, void* out, const double A[3]) {
  ZParams zp{};
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < 3; ++a) zp.gs[a] = 2.0 * pi / c->L[a];
  zp.scale = 1.0 / (double)c->N3;
  zp.comps_per_k = 2 * c->nb;
  fill_shifts(c, A, zp.shift);
  const int nbatch = 2 * c->nkb;
  const double by = 2.0 * nbatch * (double)c->N3 * 2 * sizeof(R);
  tddft_status s;
  if ((s = c->launch(KC_FFT_XY, "fft xy", [&] { return xy_pass<R>(c, in, out, nbatch, false); }, by))) return s;
  if ((s = c->launch(KC_FFT_Z, "fft z", [&] { return launch_fft_z<R>(c->st, c->N, out, nbatch, c->tw, Z_KIN, zp); }, by))) return s;
  return c->launch(KC_FFT_XY, "ifft xy", [&] { return xy_pass<R>(c, out, out, nbatch, true); }, by);
}

template <typename R> tddft_status gather(tddft_ctx* c, const void* in, const double A[3], cudaStream_t sg = nullptr) {
  if (c->natoms == 0) return TDDFT_OK;
  if (!sg) sg = c->st;
  EpiParams ep{};
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  ProjTables<R> pt = c->tables<R>();
  const double by = (double)c->n_entries * c->nkb * 2 * 2 * sizeof(R);  // psi at the sphere points
  if (c->tile) {
    const double byt = (double)c->psi_elems() * 2 * sizeof(float);  // psi read once
    return c->launch_on(sg, KC_PROJ, "projector gather (tensor cores)", [&] {
      return launch_tile_gather(sg, c->N, in, c->nk, c->nb, c->td, c->dV, ep, (const float*)c->Dmat, c->tile_part,
                                c->cbuf, c->dcbuf, c->tc_err);
    }, byt);
  }
  return c->launch_on(sg, KC_PROJ, "projector gather", [&] {
    return launch_proj_gather<R>(sg, c->N, in, c->nkb, pt, c->dV, ep, c->cbuf, c->dcbuf);
  }, by);
}

// The kinetic passes and the projector gather of one term: with a second stream the gather runs
// beside the FFT passes (fork after the previous epilogue, join before the next one).
// With the tensor-core projectors the scatter then forms V_NL psi in vnl.
template <typename R> tddft_status nl_scatter(tddft_ctx* c, const double A[3]);
template <typename R>
tddft_status kinetic_and_gather(tddft_ctx* c, const void* cur, const double A[3], bool scatter = true) {
  tddft_status s;
  if (!c->side || c->natoms == 0) {
    if ((s = kinetic<R>(c, cur, c->tmp, A))) return s;
    if ((s = gather<R>(c, cur, A))) return s;
    return scatter ? nl_scatter<R>(c, A) : TDDFT_OK;
  }
  if ((s = c->cuda(cudaEventRecord(c->ev_fork, c->st), "fork")) ||
      (s = c->cuda(cudaStreamWaitEvent(c->side, c->ev_fork, 0), "fork wait")))
    return s;
  if ((s = gather<R>(c, cur, A, c->side))) return s;
  if ((s = c->cuda(cudaEventRecord(c->ev_join, c->side), "join"))) return s;
  if ((s = kinetic<R>(c, cur, c->tmp, A))) return s;
  if ((s = c->cuda(cudaStreamWaitEvent(c->st, c->ev_join, 0), "join wait"))) return s;
  return scatter ? nl_scatter<R>(c, A) : TDDFT_OK;
}

// Tensor-core projectors: vnl = V_NL in, from the D c of the gather (main stream, after the
// join); the epilogue then adds vnl instead of running its own projector scatter.
template <typename R> tddft_status nl_scatter(tddft_ctx* c, const double A[3]) {
  if (!c->tile) return TDDFT_OK;
  EpiParams ep{};
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  const double by = (double)c->psi_elems() * 2 * sizeof(float);  // vnl written once
  return c->launch(KC_SCATTER, "projector scatter (tensor cores)", [&] {
    return launch_tile_scatter(c->st, c->N, c->vnl, c->nk, c->nb, c->td, ep, c->dcbuf, c->tc_err);
  }, by);
}
// Projector tables for the epilogue: none when the tensor cores already added V_NL psi.
template <typename R> ProjTables<R> epi_tables(const tddft_ctx* c) {
  ProjTables<R> pt = c->tables<R>();
  if (c->tile) pt.natoms = 0;
  return pt;
}

// Accumulation schedule of one series acc = sum_{i <= Ka} cf[i] T_i in the unfused recurrence:
// epilogue k has T_{k-1}, T_k and T_{k+1} in registers, so the accumulator is touched only
// when three terms are pending or T_{k+1} is its last term (one read-modify-write per three
// terms instead of one per term).  `done` is the first term not yet added; the first update
// writes without reading.  Coefficients go to cm (T_{k-1}), c0 (T_k) and c1 (T_{k+1}).
static void acc_schedule(int k, int Ka, const std::vector<cd>& cf, int& done, int& use, int& init, double* cm,
                         double* c0, double* c1) {
  use = 0;
  init = 0;
  cm[0] = cm[1] = c0[0] = c0[1] = c1[0] = c1[1] = 0.0;
  const int last = k + 1;
  if (done > Ka || last > Ka) return;
  if (last - done + 1 < 3 && last != Ka) return;
  use = 1;
  init = (done == 0);
  double* slot[3] = {cm, c0, c1};
  for (int i = done; i <= last; ++i) {
    double* d = slot[i - (k - 1)];
    d[0] = cf[i].real();
    d[1] = cf[i].imag();
  }
  done = last + 1;
}

// One Chebyshev series: T_k of H~ = (H - c)/Delta applied to `in`, accumulated with
// coefficients cf1 (orders 0..K1) into acc1 and, when acc2 is set, cf2 (0..K2) into acc2.
template <typename R>
tddft_status cheb_series(tddft_ctx* c, const void* in, const R* Vr, const double A[3], void* acc1,
                         const std::vector<cd>& cf1, int K1, void* acc2, const std::vector<cd>& cf2, int K2,
                         void* const* slots = nullptr) {
  const int K = std::max(K1, acc2 ? K2 : 0);
  EpiParams ep{};
  ep.c = 0.5 * (c->emax + c->emin);
  ep.inv_delta = 1.0 / (0.5 * (c->emax - c->emin));
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  ProjTables<R> pt = epi_tables<R>(c);
  const void* prev = in;
  const void* cur = in;
  tddft_status s;
  int done1 = 0, done2 = 0;
  // tensor-core projectors: the scatter and the epilogue run as one kernel
  const bool fuse = c->tile && c->epi_fuse && std::is_same<R, float>::value;
  for (int k = 0; k < K; ++k) {
    if ((s = kinetic_and_gather<R>(c, cur, A, !fuse))) return s;
    void* out;
    if (slots) out = slots[k + 1];
    else if (k == 0) out = c->Ta;
    else if (prev == in) out = (cur == c->Ta) ? c->Tb : c->Ta;
    else out = const_cast<void*>(prev);
    ep.mode = (k == 0) ? EPI_FIRST : EPI_RECUR;
    acc_schedule(k, K1, cf1, done1, ep.use_acc1, ep.init1, ep.am, ep.a0, ep.a1);
    if (acc2) acc_schedule(k, K2, cf2, done2, ep.use_acc2, ep.init2, ep.bm, ep.b0, ep.b1);
    else ep.use_acc2 = 0;
    const void* tkm1 = (k == 0) ? nullptr : prev;
    const double streams = 3.0 + (k == 0 ? 0.0 : 1.0) + (ep.use_acc1 ? (ep.init1 ? 1.0 : 2.0) : 0.0) +
                           (ep.use_acc2 ? (ep.init2 ? 1.0 : 2.0) : 0.0);
    const double by = streams * c->psi_elems() * 2 * sizeof(R) + 4.0 * c->N3 * sizeof(R);
    if (fuse) {
      EpiIO io;
      io.kin = (const float2*)c->tmp;
      io.Tk = (const float2*)cur;
      io.Tkm1 = (const float2*)tkm1;
      io.Tout = (float2*)out;
      io.acc1 = (float2*)acc1;
      io.acc2 = (float2*)acc2;
      io.V = (const float*)Vr;
      if ((s = c->launch(KC_EPI, "chebyshev epilogue with the tensor-core scatter", [&] {
             return launch_tile_epilogue(c->st, c->N, c->nk, c->nb, c->td, ep, c->dcbuf, c->tc_err, io);
           }, by)))
        return s;
    } else if ((s = c->launch(KC_EPI, "chebyshev epilogue", [&] {
                  return epilogue<R>(c, c->tmp, cur, tkm1, out, acc1, acc2, Vr, pt, c->dcbuf, c->nkb, ep);
                }, by))) {
      return s;
    }
    prev = cur;
    cur = out;
  }
  return TDDFT_OK;
}

// Taylor series: acc = sum_{k <= K} (-i tau H)^k / k! in.
template <typename R>
tddft_status taylor_series(tddft_ctx* c, const void* in, bool vcur, const double A[3], double tau, int K, void* acc) {
  tddft_status s = c->cuda(cudaMemcpyAsync(acc, in, c->psi_elems() * 2 * sizeof(R), cudaMemcpyDeviceToDevice, c->st),
                           "taylor init");
  if (s) return s;
  EpiParams ep{};
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  ep.mode = EPI_TAYLOR;
  ep.use_acc1 = 1;
  ProjTables<R> pt = epi_tables<R>(c);
  const R* Vr = vsel<R>(c, vcur);
  const void* cur = in;
  for (int k = 1; k <= K; ++k) {
    if ((s = kinetic_and_gather<R>(c, cur, A))) return s;
    void* out = (cur == c->Ta) ? c->Tb : c->Ta;
    ep.a1[0] = 0.0;
    ep.a1[1] = -tau / k;
    if ((s = c->launch(KC_EPI, "taylor epilogue", [&] {
           return epilogue<R>(c, c->tmp, cur, nullptr, out, acc, nullptr, Vr, pt, c->dcbuf, c->nkb, ep);
         })))
      return s;
    cur = out;
  }
  return TDDFT_OK;
}

template <typename R> tddft_status one_step(tddft_ctx* c) {
  const double t0 = c->t, t1 = c->t + c->dt;
  double A0[3], B0[3], A1[3], B1[3];
  c->fields(t0, A0, B0);
  c->fields(t1, A1, B1);
  float* Vnf = c->prec == TDDFT_FP64 ? nullptr : c->Vnewf;
  float* Vcf = c->prec == TDDFT_FP64 ? nullptr : c->Vf;
  tddft_status s;
  if (c->exp_kind != TDDFT_EXP_TAYLOR) {
    if ((s = cheb_series<R>(c, c->psi, vsel<R>(c, true), A0, c->pred, c->cf_full, c->K_full, c->phi, c->cf_half,
                            c->K_half)))
      return s;
  } else {
    if ((s = taylor_series<R>(c, c->psi, true, A0, c->dt, c->K_full, c->pred))) return s;
    if ((s = taylor_series<R>(c, c->psi, true, A0, 0.5 * c->dt, c->K_half, c->phi))) return s;
  }
  if ((s = density<R>(c, c->pred, c->rho2))) return s;
  if ((s = potential(c, c->rho2, t1, c->Vnew, Vnf))) return s;
  if ((s = window_check(c, c->Vnew))) return s;
  auto half = [&]() -> tddft_status {
    if (c->exp_kind != TDDFT_EXP_TAYLOR)
      return cheb_series<R>(c, c->phi, vsel<R>(c, false), A1, c->psi, c->cf_half, c->K_half, nullptr, c->cf_half, 0);
    return taylor_series<R>(c, c->phi, false, A1, 0.5 * c->dt, c->K_half, c->psi);
  };
  if ((s = half())) return s;
  double* rprev = c->rho2;
  double* rnext = c->rho3;
  for (int it = 0; it < c->n_sc; ++it) {
    if ((s = density<R>(c, c->psi, rnext))) return s;
    if (c->sc_tol > 0.0) {
      if ((s = c->launch(KC_OTHER, "sc diff", [&] { return launch_max_abs_diff(c->st, 4 * c->N3, rnext, rprev, c->red); })))
        return s;
      double d = 0.0;
      if ((s = c->cuda(cudaMemcpyAsync(&d, c->red, sizeof(double), cudaMemcpyDeviceToHost, c->st), "sc read"))) return s;
      if ((s = c->cuda(cudaStreamSynchronize(c->st), "sc sync"))) return s;
      if (d < c->sc_tol) break;
    }
    if ((s = potential(c, rnext, t1, c->Vnew, Vnf))) return s;
    if ((s = window_check(c, c->Vnew))) return s;
    if ((s = half())) return s;
    std::swap(rprev, rnext);
  }
  if ((s = density<R>(c, c->psi, c->rho))) return s;
  if ((s = potential(c, c->rho, t1, c->V, Vcf))) return s;
  if ((s = window_check(c, c->V))) return s;
  c->t = t1;
  return TDDFT_OK;
}

// =================================================================== discrete adjoint
// Reverse mode of one_step with the cotangent convention dL = Re sum conj(xbar) dx.  The forward
// internals of each step are recomputed from the stored psi_n with every Chebyshev term kept;
// the Chebyshev series are reversed with the Clenshaw-type recurrence
//   S_k = conj(a_k) ybar + f (H - c)/Delta S_{k+1} - S_{k+2},  f = 2 (k >= 1), 1 (k = 0),
// and dH enters through the pairs Re<S_{k+1}, f/Delta dH T_k>.

struct DevBuf {  // temporary device allocations owned by one backward call
  std::vector<void*> p;
  ~DevBuf() {
    for (void* q : p) cudaFree(q);
  }
};

template <typename T> tddft_status tmp_alloc(tddft_ctx* c, DevBuf& db, T** out, size_t bytes, const char* what) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    c->err = std::string("cudaMalloc ") + what + ": " + cudaGetErrorString(e);
    return TDDFT_ERR_OOM;
  }
  db.p.push_back(q);
  *out = (T*)q;
  return TDDFT_OK;
}

struct AdjWork {
  std::vector<void*> slots1;               // T_1..T_K1 of series 1 (index 0 unused)
  std::vector<std::vector<void*>> slots2;  // per half-step pass: T_1..T_Kh
  std::vector<void*> outs;                 // psi^(j) of pass j
  void *pred = nullptr, *phi = nullptr, *Sa = nullptr, *Sb = nullptr, *tmp2 = nullptr;
  void *PB = nullptr, *YB = nullptr, *PHIB = nullptr;
  double *rho_n = nullptr, *V_n = nullptr;
  float* Vf_n = nullptr;
  std::vector<double*> rhos, Vs;
  std::vector<float*> Vfs;
  double *gV = nullptr, *rbar = nullptr, *gvf = nullptr, *gbf = nullptr, *part = nullptr, *agrad = nullptr;
  void *cS = nullptr, *dcS = nullptr, *cT = nullptr, *dcT = nullptr;
  double* apart = nullptr;                 // projector-phase gradient partials [nkb][natoms][3]
  size_t ncoef = 0;
};

template <typename R> const R* vptr(tddft_ctx* c, double* Vd, float* Vf) {
  return c->prec == TDDFT_FP64 ? (const R*)Vd : (const R*)(const void*)Vf;
}

template <typename R>
tddft_status gather_into(tddft_ctx* c, const void* in, const double A[3], void* cb, void* dcb) {
  if (c->natoms == 0) return TDDFT_OK;
  EpiParams ep{};
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  ProjTables<R> pt = c->tables<R>();
  return c->launch(KC_PROJ, "adjoint gather", [&] {
    return launch_proj_gather<R>(c->st, c->N, in, c->nkb, pt, c->dV, ep, cb, dcb);
  });
}


// Reverse of one Chebyshev series with terms T[0..K-1]; seeds (y1, a1 up to K1), (y2, a2 up to K2).
// Accumulates the potential gradient into w.gV, the A-gradient into gA[3]; returns S_0 in *xbar.
template <typename R>
tddft_status cheb_adjoint(tddft_ctx* c, AdjWork& w, const std::vector<const void*>& T, int K, const void* y1,
                          const std::vector<cd>& a1, int K1, const void* y2, const std::vector<cd>& a2, int K2,
                          const R* Vr, const double A[3], double gA[3], void** xbar) {
  EpiParams ep{};
  ep.c = 0.5 * (c->emax + c->emin);
  ep.inv_delta = 1.0 / (0.5 * (c->emax - c->emin));
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  ZParams zp{};
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < 3; ++a) zp.gs[a] = 2.0 * pi / c->L[a];
  zp.scale = 1.0 / (double)c->N3;
  zp.comps_per_k = 2 * c->nb;
  fill_shifts(c, A, zp.shift);
  ProjTables<R> pt = c->tables<R>();
  const int nbatch = 2 * c->nkb;
  const size_t n = c->psi_elems();
  tddft_status s;
  auto coef = [&](int k, double* ca, double* cb, int* u1, int* u2) {
    *u1 = (y1 && k <= K1) ? 1 : 0;
    *u2 = (y2 && k <= K2) ? 1 : 0;
    ca[0] = ca[1] = cb[0] = cb[1] = 0.0;
    if (*u1) { ca[0] = a1[k].real(); ca[1] = -a1[k].imag(); }
    if (*u2) { cb[0] = a2[k].real(); cb[1] = -a2[k].imag(); }
  };
  if ((s = c->cuda(cudaMemsetAsync(w.agrad, 0, (3 * (size_t)c->nkb + 3) * sizeof(double), c->st), "agrad reset")))
    return s;
  double* agk = w.agrad + 3 * (size_t)c->nkb;  // kinetic part
  {
    double ca[2], cb[2];
    int u1, u2;
    coef(K, ca, cb, &u1, &u2);
    if ((s = c->launch(KC_OTHER, "adjoint seed", [&] {
           return launch_seed<R>(c->st, n, u1 ? y1 : nullptr, ca, u2 ? y2 : nullptr, cb, w.Sa);
         })))
      return s;
  }
  void* cur = w.Sa;
  void* prev2 = nullptr;
  for (int k = K - 1; k >= 0; --k) {
    const void* Tk = T[k];
    const double f = (k >= 1 ? 2.0 : 1.0) * ep.inv_delta;
    if ((s = c->launch(KC_OTHER, "grad V", [&] { return launch_grad_v<R>(c->st, c->N3, c->nkb, cur, Tk, f, w.gV, c->rho_part); })))
      return s;
    if ((s = c->launch(KC_FFT_XY, "adj fft xy", [&] { return xy_pass<R>(c, cur, c->tmp, nbatch, false); }))) return s;
    if ((s = c->launch(KC_FFT_XY, "adj fft xy T", [&] { return xy_pass<R>(c, Tk, w.tmp2, nbatch, false); }))) return s;
    if ((s = c->launch(KC_FFT_Z, "adj fft z current", [&] {
           return launch_fft_z_current<R>(c->st, c->N, c->tmp, w.tmp2, nbatch, c->tw, zp, w.part);
         })))
      return s;
    if ((s = c->launch(KC_OTHER, "adj current sum", [&] {
           return launch_accum_parts(c->st, (size_t)nbatch * c->N, w.part, f / (double)c->N3, agk);
         })))
      return s;
    if ((s = c->launch(KC_FFT_XY, "adj ifft xy", [&] { return xy_pass<R>(c, c->tmp, c->tmp, nbatch, true); }))) return s;
    if (c->natoms > 0) {
      if ((s = gather_into<R>(c, cur, A, w.cS, w.dcS)) || (s = gather_into<R>(c, Tk, A, w.cT, w.dcT))) return s;
      if ((s = c->launch(KC_PROJ, "adj nl agrad", [&] {
             return launch_nl_agrad_fused<R>(c->st, c->N, cur, Tk, c->nkb, pt, ep, w.dcS, w.dcT, f, w.apart, w.agrad);
           })))
        return s;
    }
    void* out = prev2 ? prev2 : (cur == w.Sa ? w.Sb : w.Sa);
    double ca[2], cb[2];
    int u1, u2;
    coef(k, ca, cb, &u1, &u2);
    ep.mode = (k >= 1) ? EPI_ADJ : EPI_ADJ0;
    ep.use_acc1 = u1;
    ep.use_acc2 = u2;
    ep.a1[0] = ca[0]; ep.a1[1] = ca[1];
    ep.b1[0] = cb[0]; ep.b1[1] = cb[1];
    const void* s2 = prev2;
    if ((s = c->launch(KC_EPI, "adjoint epilogue", [&] {
           return epilogue<R>(c, c->tmp, cur, s2, out, const_cast<void*>(y1), const_cast<void*>(y2), Vr,
                                     pt, w.dcS, c->nkb, ep);
         })))
      return s;
    prev2 = cur;
    cur = out;
  }
  *xbar = cur;
  std::vector<double> h(3 * (size_t)c->nkb + 3);
  if ((s = c->cuda(cudaMemcpyAsync(h.data(), w.agrad, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st), "agrad read")))
    return s;
  if ((s = c->cuda(cudaStreamSynchronize(c->st), "agrad sync"))) return s;
  for (int kb = 0; kb < c->nkb; ++kb)
    for (int a = 0; a < 3; ++a) gA[a] += h[3 * kb + a];
  for (int a = 0; a < 3; ++a) gA[a] += h[3 * (size_t)c->nkb + a];
  return TDDFT_OK;
}

// rhobar and dL/dB from w.gV (cotangent of V_v) at density rho: XC Jacobian-transpose,
// Hartree (symmetric convolution) and the uniform Zeeman coupling mu_B B.sigma.
tddft_status potential_adjoint(tddft_ctx* c, AdjWork& w, const double* rho, double gB[3]) {
  tddft_status s;
  ZParams zp{};
  const double pi = 3.14159265358979323846;
  for (int a = 0; a < 3; ++a) zp.gs[a] = 2.0 * pi / c->L[a];
  zp.scale = 1.0 / (double)c->N3;
  if ((s = c->launch(KC_POT, "xc adjoint", [&] { return launch_xc_adjoint(c->st, c->N3, rho, w.gV, c->xc, w.rbar, w.gvf, w.gbf); }))) return s;
  if ((s = c->launch(KC_POT, "hartree adj in", [&] { return launch_real_field_to_complex(c->st, c->N3, w.gvf, c->hart); }))) return s;
  if ((s = c->launch(KC_POT, "hartree adj xy", [&] { return launch_fft_xy<double>(c->st, c->N, c->hart, c->hart, 1, c->tw64, false); }))) return s;
  if ((s = c->launch(KC_POT, "hartree adj z", [&] { return launch_fft_z<double>(c->st, c->N, c->hart, 1, c->tw64, Z_POISSON, zp); }))) return s;
  if ((s = c->launch(KC_POT, "hartree adj ixy", [&] { return launch_fft_xy<double>(c->st, c->N, c->hart, c->hart, 1, c->tw64, true); }))) return s;
  if ((s = c->launch(KC_POT, "hartree adj add", [&] { return launch_add_hartree_adjoint(c->st, c->N3, c->hart, w.rbar); }))) return s;
  if ((s = c->launch(KC_POT, "b sums", [&] { return launch_sum3(c->st, c->N3, w.gbf, c->red); }))) return s;
  double h[3];
  if ((s = c->cuda(cudaMemcpyAsync(h, c->red, sizeof(h), cudaMemcpyDeviceToHost, c->st), "b read"))) return s;
  if ((s = c->cuda(cudaStreamSynchronize(c->st), "b sync"))) return s;
  for (int a = 0; a < 3; ++a) gB[a] += 0.5 * h[a];  // mu_B = 1/2
  return TDDFT_OK;
}

template <typename R>
tddft_status density_adj(tddft_ctx* c, const void* psi, const double* rbar, const void* add, void* out) {
  return c->launch(KC_DENS, "density adjoint", [&] {
    return launch_density_adjoint<R>(c->st, c->N3, c->nkb, psi, rbar, c->wf_d, add, out);
  });
}

// w.PB holds psibar_{n+1} on entry and psibar_n on exit; gradients with respect to A, B at
// t0 and t0 + dt are added to gA0, gB0, gA1, gB1.
template <typename R>
tddft_status adjoint_step(tddft_ctx* c, AdjWork& w, const void* psi_n, double t0, double gA0[3], double gB0[3],
                          double gA1[3], double gB1[3]) {
  const double t1 = t0 + c->dt;
  double A0[3], B0[3], A1[3], B1[3];
  c->fields(t0, A0, B0);
  c->fields(t1, A1, B1);
  const bool f64 = c->prec == TDDFT_FP64;
  const int K1 = std::max(c->K_full, c->K_half), Kh = c->K_half;
  const size_t n = c->psi_elems();
  tddft_status s;
  // ---- recompute the step, keeping every term
  if ((s = density<R>(c, psi_n, w.rho_n)) || (s = potential(c, w.rho_n, t0, w.V_n, f64 ? nullptr : w.Vf_n))) return s;
  if ((s = cheb_series<R>(c, psi_n, vptr<R>(c, w.V_n, w.Vf_n), A0, w.pred, c->cf_full, c->K_full, w.phi, c->cf_half,
                          c->K_half, w.slots1.data())))
    return s;
  const void* src = w.pred;
  for (int j = 0; j <= c->n_sc; ++j) {
    if ((s = density<R>(c, src, w.rhos[j])) || (s = potential(c, w.rhos[j], t1, w.Vs[j], f64 ? nullptr : w.Vfs[j]))) return s;
    if ((s = cheb_series<R>(c, w.phi, vptr<R>(c, w.Vs[j], w.Vfs[j]), A1, w.outs[j], c->cf_half, Kh, nullptr, c->cf_half,
                            0, w.slots2[j].data())))
      return s;
    src = w.outs[j];
  }
  // ---- reverse through the half-step passes at t + dt
  const void* ybar = w.PB;
  bool have_phibar = false;
  for (int j = c->n_sc; j >= 0; --j) {
    if ((s = c->cuda(cudaMemsetAsync(w.gV, 0, 4 * c->N3 * sizeof(double), c->st), "gV reset"))) return s;
    std::vector<const void*> T(Kh);
    T[0] = w.phi;
    for (int k = 1; k < Kh; ++k) T[k] = w.slots2[j][k];
    void* xbar = nullptr;
    if ((s = cheb_adjoint<R>(c, w, T, Kh, ybar, c->cf_half, Kh, nullptr, c->cf_half, -1, vptr<R>(c, w.Vs[j], w.Vfs[j]),
                             A1, gA1, &xbar)))
      return s;
    const double one[2] = {1.0, 0.0};
    if ((s = c->launch(KC_OTHER, "phibar", [&] {
           return launch_seed<R>(c->st, n, have_phibar ? w.PHIB : nullptr, one, xbar, one, w.PHIB);
         })))
      return s;
    have_phibar = true;
    if ((s = potential_adjoint(c, w, w.rhos[j], gB1))) return s;
    const void* srcj = (j == 0) ? w.pred : w.outs[j - 1];
    if ((s = density_adj<R>(c, srcj, w.rbar, nullptr, w.YB))) return s;
    ybar = w.YB;
  }
  // ---- reverse through series 1 (shared terms for psi~ and phi) at t
  if ((s = c->cuda(cudaMemsetAsync(w.gV, 0, 4 * c->N3 * sizeof(double), c->st), "gV reset"))) return s;
  std::vector<const void*> T(K1);
  T[0] = psi_n;
  for (int k = 1; k < K1; ++k) T[k] = w.slots1[k];
  void* xbar = nullptr;
  if ((s = cheb_adjoint<R>(c, w, T, K1, w.YB, c->cf_full, c->K_full, w.PHIB, c->cf_half, c->K_half,
                           vptr<R>(c, w.V_n, w.Vf_n), A0, gA0, &xbar)))
    return s;
  if ((s = potential_adjoint(c, w, w.rho_n, gB0))) return s;
  return density_adj<R>(c, psi_n, w.rbar, xbar, w.PB);
}

// Lerp weights of the field table at time tt, matching field_at.
void table_weights(const tddft_ctx* c, double tt, int* j0, double* w0, int* j1, double* w1) {
  const int nt = (int)c->ft.size();
  *j0 = *j1 = 0;
  *w0 = *w1 = 0.0;
  if (nt == 0) return;
  if (tt <= c->ft[0] || nt == 1) { *j0 = 0; *w0 = 1.0; return; }
  if (tt >= c->ft[nt - 1]) { *j0 = nt - 1; *w0 = 1.0; return; }
  const int j = (int)(std::upper_bound(c->ft.begin(), c->ft.end(), tt) - c->ft.begin());
  const double a = (tt - c->ft[j - 1]) / (c->ft[j] - c->ft[j - 1]);
  *j0 = j - 1; *w0 = 1.0 - a; *j1 = j; *w1 = a;
}

void add_table(const tddft_ctx* c, double tt, const double gA[3], const double gB[3], double* dA, double* dB) {
  int j0, j1;
  double w0, w1;
  table_weights(c, tt, &j0, &w0, &j1, &w1);
  if (c->ft.empty()) return;
  for (int a = 0; a < 3; ++a) {
    dA[3 * j0 + a] += w0 * gA[a];
    dB[3 * j0 + a] += w0 * gB[a];
    if (w1 != 0.0) {
      dA[3 * j1 + a] += w1 * gA[a];
      dB[3 * j1 + a] += w1 * gB[a];
    }
  }
}

template <typename R>
tddft_status do_backward(tddft_ctx* c, int nsteps, int ckpt, const double* dL_drho, double* loss, double* dA,
                         double* dB) {
  if (c->exp_kind == TDDFT_EXP_TAYLOR || c->sc_tol > 0.0)
    return c->fail(TDDFT_ERR_UNSUPPORTED, "backward needs Chebyshev or Crank-Nicolson exponentials and sc_tol = 0");
  {
    const size_t smem = (size_t)(c->N + 2 * c->N * (c->N + 1)) * 2 * sizeof(R) + 24 * sizeof(double);
    if (smem > 227 * 1024) return c->fail(TDDFT_ERR_UNSUPPORTED, "backward: grid too large for the adjoint z pass");
  }
  if (ckpt < 1) ckpt = nsteps > 0 ? nsteps : 1;
  const size_t nt = c->ft.size();
  for (size_t i = 0; i < 3 * nt; ++i) {
    if (dA) dA[i] = 0.0;
    if (dB) dB[i] = 0.0;
  }
  std::vector<double> gAt(3 * std::max<size_t>(nt, 1), 0.0), gBt(3 * std::max<size_t>(nt, 1), 0.0);
  DevBuf db;
  AdjWork w;
  const size_t pb = c->psi_elems() * 2 * sizeof(R);
  const size_t N3 = c->N3;
  const int K1 = std::max(c->K_full, c->K_half), Kh = c->K_half;
  tddft_status s;
  w.slots1.assign(K1 + 1, nullptr);
  for (int k = 1; k <= K1; ++k)
    if ((s = tmp_alloc(c, db, &w.slots1[k], pb, "adjoint T1"))) return s;
  w.slots2.assign(c->n_sc + 1, std::vector<void*>(Kh + 1, nullptr));
  w.outs.assign(c->n_sc + 1, nullptr);
  w.rhos.assign(c->n_sc + 1, nullptr);
  w.Vs.assign(c->n_sc + 1, nullptr);
  w.Vfs.assign(c->n_sc + 1, nullptr);
  for (int j = 0; j <= c->n_sc; ++j) {
    for (int k = 1; k <= Kh; ++k)
      if ((s = tmp_alloc(c, db, &w.slots2[j][k], pb, "adjoint T2"))) return s;
    if ((s = tmp_alloc(c, db, &w.outs[j], pb, "adjoint out")) || (s = tmp_alloc(c, db, &w.rhos[j], 4 * N3 * 8, "adj rho")) ||
        (s = tmp_alloc(c, db, &w.Vs[j], 4 * N3 * 8, "adj V")))
      return s;
    if (c->prec != TDDFT_FP64 && (s = tmp_alloc(c, db, &w.Vfs[j], 4 * N3 * 4, "adj Vf"))) return s;
  }
  if ((s = tmp_alloc(c, db, &w.pred, pb, "adj pred")) || (s = tmp_alloc(c, db, &w.phi, pb, "adj phi")) ||
      (s = tmp_alloc(c, db, &w.Sa, pb, "adj Sa")) || (s = tmp_alloc(c, db, &w.Sb, pb, "adj Sb")) ||
      (s = tmp_alloc(c, db, &w.tmp2, pb, "adj tmp2")) || (s = tmp_alloc(c, db, &w.PB, pb, "adj PB")) ||
      (s = tmp_alloc(c, db, &w.YB, pb, "adj YB")) || (s = tmp_alloc(c, db, &w.PHIB, pb, "adj PHIB")) ||
      (s = tmp_alloc(c, db, &w.rho_n, 4 * N3 * 8, "adj rho_n")) || (s = tmp_alloc(c, db, &w.V_n, 4 * N3 * 8, "adj V_n")) ||
      (s = tmp_alloc(c, db, &w.gV, 4 * N3 * 8, "adj gV")) || (s = tmp_alloc(c, db, &w.rbar, 4 * N3 * 8, "adj rbar")) ||
      (s = tmp_alloc(c, db, &w.gvf, N3 * 8, "adj gvf")) || (s = tmp_alloc(c, db, &w.gbf, 3 * N3 * 8, "adj gbf")) ||
      (s = tmp_alloc(c, db, &w.part, (size_t)2 * c->nkb * c->N * 3 * 8, "adj part")) ||
      (s = tmp_alloc(c, db, &w.agrad, (3 * (size_t)c->nkb + 3) * 8, "adj agrad")))
    return s;
  if (c->prec != TDDFT_FP64 && (s = tmp_alloc(c, db, &w.Vf_n, 4 * N3 * 4, "adj Vf_n"))) return s;
  w.ncoef = (size_t)c->nkb * std::max(1, c->natoms) * 2 * c->nlm;
  const size_t cb = w.ncoef * 2 * sizeof(R);
  if ((s = tmp_alloc(c, db, &w.cS, cb, "cS")) || (s = tmp_alloc(c, db, &w.dcS, cb, "dcS")) ||
      (s = tmp_alloc(c, db, &w.apart, (size_t)c->nkb * std::max(c->natoms, 1) * 3 * 8, "agrad parts")) ||
      (s = tmp_alloc(c, db, &w.cT, cb, "cT")) || (s = tmp_alloc(c, db, &w.dcT, cb, "dcT")))
    return s;
  const int nck = (nsteps + ckpt - 1) / ckpt;
  std::vector<void*> ck(std::max(nck, 1), nullptr), seg(ckpt, nullptr);
  for (int i = 0; i < nck; ++i)
    if ((s = tmp_alloc(c, db, &ck[i], pb, "checkpoint"))) return s;
  for (int i = 0; i < ckpt; ++i)
    if ((s = tmp_alloc(c, db, &seg[i], pb, "segment"))) return s;
  // ---- forward with checkpoints
  std::vector<double> times(nsteps + 1);
  times[0] = c->t;
  for (int n = 0; n < nsteps; ++n) {
    if (n % ckpt == 0 && (s = c->cuda(cudaMemcpyAsync(ck[n / ckpt], c->psi, pb, cudaMemcpyDeviceToDevice, c->st), "ckpt")))
      return s;
    if ((s = one_step<R>(c))) return s;
    times[n + 1] = c->t;
  }
  // ---- loss and seed
  std::vector<double> rho_h(4 * N3);
  if ((s = c->cuda(cudaMemcpyAsync(rho_h.data(), c->rho, rho_h.size() * 8, cudaMemcpyDeviceToHost, c->st), "rho read")) ||
      (s = c->cuda(cudaStreamSynchronize(c->st), "rho sync")))
    return s;
  double L = 0.0;
  for (size_t i = 0; i < 4 * N3; ++i) L += dL_drho[i] * rho_h[i];
  if (loss) *loss = L;
  void* final_psi = nullptr;
  if ((s = tmp_alloc(c, db, &final_psi, pb, "final psi")) ||
      (s = c->cuda(cudaMemcpyAsync(final_psi, c->psi, pb, cudaMemcpyDeviceToDevice, c->st), "final copy")) ||
      (s = c->cuda(cudaMemcpyAsync(w.rbar, dL_drho, 4 * N3 * 8, cudaMemcpyHostToDevice, c->st), "seed upload")) ||
      (s = density_adj<R>(c, c->psi, w.rbar, nullptr, w.PB)))
    return s;
  const double t_final = c->t;
  // ---- reverse over checkpoint segments
  for (int sg = nck - 1; sg >= 0; --sg) {
    const int s0 = sg * ckpt, s1 = std::min(nsteps, s0 + ckpt);
    if ((s = c->cuda(cudaMemcpyAsync(c->psi, ck[sg], pb, cudaMemcpyDeviceToDevice, c->st), "restore")) ||
        (s = c->cuda(cudaMemcpyAsync(seg[0], ck[sg], pb, cudaMemcpyDeviceToDevice, c->st), "seg0")))
      return s;
    c->t = times[s0];
    float* Vcf = c->prec == TDDFT_FP64 ? nullptr : c->Vf;
    if ((s = density<R>(c, c->psi, c->rho)) || (s = potential(c, c->rho, c->t, c->V, Vcf))) return s;
    for (int n = s0; n < s1 - 1; ++n) {
      if ((s = one_step<R>(c))) return s;
      if ((s = c->cuda(cudaMemcpyAsync(seg[n - s0 + 1], c->psi, pb, cudaMemcpyDeviceToDevice, c->st), "seg copy"))) return s;
    }
    for (int n = s1 - 1; n >= s0; --n) {
      double gA0[3] = {0, 0, 0}, gB0[3] = {0, 0, 0}, gA1[3] = {0, 0, 0}, gB1[3] = {0, 0, 0};
      if ((s = adjoint_step<R>(c, w, seg[n - s0], times[n], gA0, gB0, gA1, gB1))) return s;
      add_table(c, times[n], gA0, gB0, gAt.data(), gBt.data());
      add_table(c, times[n] + c->dt, gA1, gB1, gAt.data(), gBt.data());
    }
  }
  // ---- restore the forward end state
  if ((s = c->cuda(cudaMemcpyAsync(c->psi, final_psi, pb, cudaMemcpyDeviceToDevice, c->st), "final restore"))) return s;
  c->t = t_final;
  {
    float* Vcf = c->prec == TDDFT_FP64 ? nullptr : c->Vf;
    if ((s = density<R>(c, c->psi, c->rho)) || (s = potential(c, c->rho, c->t, c->V, Vcf))) return s;
  }
  if ((s = c->cuda(cudaStreamSynchronize(c->st), "backward sync"))) return s;
  for (size_t i = 0; i < 3 * nt; ++i) {
    if (dA) dA[i] = gAt[i];
    if (dB) dB[i] = gBt[i];
  }
  return TDDFT_OK;
}

void set_orders(tddft_ctx* c) {
  const double dlt = 0.5 * (c->emax - c->emin);
  const double cc = 0.5 * (c->emax + c->emin);
  if (c->exp_kind == TDDFT_EXP_CHEBYSHEV) {
    double tol = c->cheb_tol > 0 ? c->cheb_tol : (c->prec == TDDFT_FP64 ? 1e-16 : 1e-9);
    if (c->exp_order > 0) {
      c->K_full = c->K_half = c->exp_order;
    } else {
      c->K_full = chebyshev_order(c->dt * dlt, tol);
      c->K_half = chebyshev_order(0.5 * c->dt * dlt, tol);
    }
    auto coefs = [&](double tau, int K) {
      std::vector<cd> a(K + 1);
      auto J = bessel_j(K, tau * dlt);
      const cd ph = std::exp(cd(0.0, -tau * cc));
      cd mi(1.0, 0.0);
      for (int k = 0; k <= K; ++k) {
        a[k] = (k == 0 ? 1.0 : 2.0) * mi * J[k] * ph;
        mi *= cd(0.0, -1.0);
      }
      return a;
    };
    c->cf_full = coefs(c->dt, c->K_full);
    c->cf_half = coefs(0.5 * c->dt, c->K_half);
  } else if (c->exp_kind == TDDFT_EXP_CRANK_NICOLSON) {
    // Chebyshev coefficients of the Cayley transform f(E) = (1 - i tau E/2) / (1 + i tau E/2) on
    // [emin, emax]: a_k = (2 - delta_k0)/Q sum_j f(c + Delta cos th_j) cos(k th_j), th_j = pi (j + 1/2)/Q
    // (Gauss-Chebyshev).  f has its pole at E = 2i/tau, off the window, so a_k decays
    // geometrically; Q = 4096 nodes leave an aliasing error far below the truncation.
    const double tol = c->cheb_tol > 0 ? c->cheb_tol : (c->prec == TDDFT_FP64 ? 1e-16 : 1e-9);
    const double pi = 3.14159265358979323846;
    const int Q = 4096, KM = Q / 2;
    auto cn = [&](double tau, int& K) {
      std::vector<cd> fv(Q);
      std::vector<double> th(Q);
      for (int j = 0; j < Q; ++j) {
        th[j] = pi * (j + 0.5) / Q;
        const double E = cc + dlt * std::cos(th[j]);
        fv[j] = cd(1.0, -0.5 * tau * E) / cd(1.0, 0.5 * tau * E);
      }
      std::vector<cd> a(KM);
      for (int k = 0; k < KM; ++k) {
        cd sum = 0.0;
        for (int j = 0; j < Q; ++j) sum += fv[j] * std::cos(k * th[j]);
        a[k] = (k == 0 ? 1.0 : 2.0) / Q * sum;
      }
      if (c->exp_order > 0) {
        K = std::min(c->exp_order, KM - 1);
      } else {
        K = 0;
        for (int k = KM - 1; k >= 0; --k)
          if (std::abs(a[k]) >= tol) { K = k; break; }
      }
      a.resize(K + 1);
      return a;
    };
    c->cf_full = cn(c->dt, c->K_full);
    c->cf_half = cn(0.5 * c->dt, c->K_half);
  } else {
    c->K_full = c->K_half = c->exp_order > 0 ? c->exp_order : 4;
  }
}

// Device address of page-locked host memory (cudaHostAlloc, cudaHostRegister), through which a
// kernel reads or writes it directly (NVLink-C2C on Grace systems); null for pageable memory,
// which is staged through device buffers.
const void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (at.type == cudaMemoryTypeHost && at.devicePointer) ? at.devicePointer : nullptr;
}

// complex64 spinors in: a plain copy for FP32-mixed handles, an exact widening for FP64 ones
// (through the mapped address of page-locked memory, or staged in the work array Ta).
tddft_status load_states_c64(tddft_ctx* c, const void* psi, int on_device) {
  const size_t n = c->psi_elems();
  if (c->prec != TDDFT_FP64)
    return c->cuda(cudaMemcpyAsync(c->psi, psi, n * sizeof(float2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st),
                   "set_states_c64 copy");
  const void* src = on_device ? psi : mapped_host(psi);
  tddft_status s;
  if (!src) {
    if ((s = c->cuda(cudaMemcpyAsync(c->Ta, psi, n * sizeof(float2), cudaMemcpyHostToDevice, c->st), "set_states_c64 stage")))
      return s;
    src = c->Ta;
  }
  return c->launch(KC_OTHER, "widen in", [&] { return launch_convert_out<float>(c->st, n, src, (double2*)c->psi); });
}

tddft_status store_states_c64(tddft_ctx* c, void* out, int on_device) {
  const size_t n = c->psi_elems();
  tddft_status s;
  if (c->prec != TDDFT_FP64) {
    if ((s = c->cuda(cudaMemcpyAsync(out, c->psi, n * sizeof(float2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st),
                     "get_states_c64 copy")))
      return s;
  } else if (void* dst = on_device ? out : const_cast<void*>(mapped_host(out))) {
    if ((s = c->launch(KC_OTHER, "narrow out", [&] { return launch_convert_in<float>(c->st, n, (const double2*)c->psi, dst); }))) return s;
  } else {
    if ((s = c->launch(KC_OTHER, "narrow out", [&] { return launch_convert_in<float>(c->st, n, (const double2*)c->psi, c->Ta); })) ||
        (s = c->cuda(cudaMemcpyAsync(out, c->Ta, n * sizeof(float2), cudaMemcpyDeviceToHost, c->st), "get_states_c64 stage")))
      return s;
  }
  return c->cuda(cudaStreamSynchronize(c->st), "get_states_c64 sync");
}

template <typename R> tddft_status do_set_states(tddft_ctx* c, const void* psi, int on_device, double t0, bool c64 = false) {
  const size_t n = c->psi_elems();
  tddft_status s;
  if (c64) {
    if ((s = load_states_c64(c, psi, on_device))) return s;
  } else if (c->prec == TDDFT_FP64) {
    if ((s = c->cuda(cudaMemcpyAsync(c->psi, psi, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st), "set_states copy"))) return s;
  } else if (const void* src = on_device ? psi : mapped_host(psi)) {
    if ((s = c->launch(KC_OTHER, "convert in", [&] { return launch_convert_in<R>(c->st, n, (const double2*)src, c->psi); }))) return s;
  } else {
    for (size_t off = 0; off < n; off += c->stage_elems) {
      const size_t m = std::min(c->stage_elems, n - off);
      if ((s = c->cuda(cudaMemcpyAsync(c->stage, (const double2*)psi + off, m * sizeof(double2), cudaMemcpyHostToDevice, c->st), "set_states stage"))) return s;
      if ((s = c->launch(KC_OTHER, "convert in", [&] { return launch_convert_in<R>(c->st, m, c->stage, (float2*)c->psi + off); }))) return s;
    }
  }
  c->t = t0;
  if ((s = density<R>(c, c->psi, c->rho))) return s;
  float* Vcf = c->prec == TDDFT_FP64 ? nullptr : c->Vf;
  if ((s = potential(c, c->rho, t0, c->V, Vcf))) return s;
  // spectral window (reading: extrema of the potential, kinetic maximum, projector bound, 5 % margin)
  double Atab[3], Btab[3];
  c->kin_max = 0.0;
  if (c->ft.empty()) {
    Atab[0] = Atab[1] = Atab[2] = 0.0;
    for (int k = 0; k < c->nk; ++k) c->kin_max = std::max(c->kin_max, c->kinetic_max_for(&c->kpts[3 * k]));
  } else {
    for (size_t j = 0; j < c->ft.size(); ++j)
      for (int k = 0; k < c->nk; ++k) {
        double sft[3];
        for (int a = 0; a < 3; ++a) sft[a] = c->kpts[3 * k + a] + c->fA[3 * j + a];
        c->kin_max = std::max(c->kin_max, c->kinetic_max_for(sft));
      }
  }
  (void)Atab; (void)Btab;
  if (c->emin_user == 0.0 && c->emax_user == 0.0) {
    double ext[3];
    if ((s = c->launch(KC_OTHER, "window extrema", [&] { return launch_window_extrema(c->st, c->N3, c->V, c->red_part, c->red); })) ||
        (s = c->cuda(cudaMemcpyAsync(ext, c->red, sizeof(ext), cudaMemcpyDeviceToHost, c->st), "window read")) ||
        (s = c->cuda(cudaStreamSynchronize(c->st), "window sync")))
      return s;
    const double vmin = ext[0], vmax = ext[1], bmax = ext[2];
    double emin = vmin - bmax - c->nl_bound, emax = vmax + bmax + c->kin_max + c->nl_bound;
    const double w = emax - emin;
    c->emin = emin - 0.025 * w;
    c->emax = emax + 0.025 * w;
  } else {
    c->emin = c->emin_user;
    c->emax = c->emax_user;
  }
  set_orders(c);
  if ((s = c->cuda(cudaMemsetAsync(c->flag, 0, sizeof(int), c->st), "flag reset"))) return s;
  if ((s = window_check(c, c->V))) return s;
  c->have_states = true;
  return TDDFT_OK;
}

template <typename R> tddft_status do_get_states(tddft_ctx* c, void* out, int on_device) {
  const size_t n = c->psi_elems();
  tddft_status s;
  if (c->prec == TDDFT_FP64) {
    if ((s = c->cuda(cudaMemcpyAsync(out, c->psi, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st), "get_states copy"))) return s;
  } else if (void* dst = on_device ? out : const_cast<void*>(mapped_host(out))) {
    if ((s = c->launch(KC_OTHER, "convert out", [&] { return launch_convert_out<R>(c->st, n, c->psi, (double2*)dst); }))) return s;
  } else {
    for (size_t off = 0; off < n; off += c->stage_elems) {
      const size_t m = std::min(c->stage_elems, n - off);
      if ((s = c->launch(KC_OTHER, "convert out", [&] { return launch_convert_out<R>(c->st, m, (const float2*)c->psi + off, c->stage); }))) return s;
      if ((s = c->cuda(cudaMemcpyAsync((double2*)out + off, c->stage, m * sizeof(double2), cudaMemcpyDeviceToHost, c->st), "get_states stage"))) return s;
      if ((s = c->cuda(cudaStreamSynchronize(c->st), "get_states sync"))) return s;
    }
  }
  return c->cuda(cudaStreamSynchronize(c->st), "get_states sync");
}

template <typename R> tddft_status do_observables(tddft_ctx* c, double* n, double* m, double* E, double* M, double* norms) {
  tddft_status s;
  double A[3], B[3];
  c->fields(c->t, A, B);
  const int nkb = c->nkb;
  double* dots = c->red + 16;  // [nkb][2] then [nkb][2] then [nkb]
  double* kdots = dots + 2 * nkb;
  double* nle = kdots + 2 * nkb;
  if ((s = c->launch(KC_OTHER, "norms", [&] { return launch_band_dot<R>(c->st, 2 * c->N3, nkb, c->psi, c->psi, dots, c->red_part); }))) return s;
  // the kinetic and non-local energies only enter E: without E their passes are skipped
  if (E && (s = kinetic<R>(c, c->psi, c->tmp, A))) return s;
  if (E && (s = c->launch(KC_OTHER, "kinetic dot", [&] { return launch_band_dot<R>(c->st, 2 * c->N3, nkb, c->psi, c->tmp, kdots, c->red_part); }))) return s;
  if (E && c->natoms > 0) {
    if ((s = gather<R>(c, c->psi, A))) return s;
    if ((s = c->launch(KC_OTHER, "nl energy", [&] { return launch_nl_energy<R>(c->st, nkb, c->natoms * 2 * c->nlm, c->cbuf, c->dcbuf, nle); }))) return s;
  }
  if ((s = c->launch(KC_OTHER, "field sums", [&] {
         return launch_field_sums(c->st, c->N3, c->rho, c->vloc, c->vH, c->exc, c->vxc4, c->V, B, c->red, c->red_part);
       })))
    return s;
  std::vector<double> h(16 + 5 * nkb, 0.0);
  int flag = 0, tcflag = 0;
  if ((s = c->cuda(cudaMemcpyAsync(h.data(), c->red, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->st), "obs read"))) return s;
  if ((s = c->cuda(cudaMemcpyAsync(&flag, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st), "flag read"))) return s;
  if ((s = c->cuda(cudaMemcpyAsync(&tcflag, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->st), "tc flag read"))) return s;
  if (n || m) {
    // n and m are formed on the device in the step scratch rho2 (free between steps) and copied
    // straight into the caller's arrays
    const size_t N3 = c->N3;
    if ((s = c->launch(KC_OTHER, "n, m", [&] { return launch_nm_from_rho(c->st, N3, c->rho, c->rho2); }))) return s;
    if (n && (s = c->cuda(cudaMemcpyAsync(n, c->rho2, N3 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "n read")))
      return s;
    if (m && (s = c->cuda(cudaMemcpyAsync(m, c->rho2 + N3, 3 * N3 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "m read")))
      return s;
  }
  if ((s = c->cuda(cudaStreamSynchronize(c->st), "obs sync"))) return s;
  double ekin = 0, enl = 0;
  bool bad = h[9] != 0.0;
  for (int kb = 0; kb < nkb; ++kb) {
    const double w = c->wf[kb];
    const double nr = h[16 + 2 * kb] * c->dV;
    if (norms) norms[kb] = nr;
    if (!std::isfinite(nr)) bad = true;
    ekin += w * h[16 + 2 * nkb + 2 * kb] * c->dV;
    if (c->natoms > 0) enl += w * h[16 + 4 * nkb + kb];
  }
  if (E) {
    E[TDDFT_E_KIN] = ekin;
    E[TDDFT_E_NL] = enl;
    E[TDDFT_E_LOC] = h[0] * c->dV;
    E[TDDFT_E_H] = 0.5 * h[1] * c->dV;
    E[TDDFT_E_XC] = h[2] * c->dV;
    E[TDDFT_E_Z] = 0.5 * h[7] * c->dV;
    E[TDDFT_E_TOTAL] = E[0] + E[1] + E[2] + E[3] + E[4] + E[5];
    E[TDDFT_E_TIME] = c->t;
    E[TDDFT_E_XC_POT] = h[8] * c->dV;
    E[TDDFT_E_NELEC] = h[6] * c->dV;
  }
  if (M)
    for (int a = 0; a < 3; ++a) M[a] = h[3 + a] * c->dV;
  if (tcflag & 1) return c->fail(TDDFT_ERR_CUDA, "a tensor-core projector wait exceeded its iteration limit");
  if (tcflag & 2) return c->fail(TDDFT_ERR_CUDA, "a bulk-copy wait of an FFT pass exceeded its iteration limit");
  if (bad) return c->fail(TDDFT_ERR_DIVERGED, "non-finite density or norm");
  if (flag) return c->fail(TDDFT_ERR_BOUND, "potential left the Chebyshev spectral window");
  return TDDFT_OK;
}

template <typename R> tddft_status do_apply_h(tddft_ctx* c, const void* in, void* out, int on_device) {
  const size_t n = c->psi_elems();
  tddft_status s;
  double A[3], B[3];
  c->fields(c->t, A, B);
  // stage the input into Ta (precision R)
  if (c->prec == TDDFT_FP64) {
    if ((s = c->cuda(cudaMemcpyAsync(c->Ta, in, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st), "apply_h in"))) return s;
  } else if (on_device) {
    if ((s = c->launch(KC_OTHER, "convert in", [&] { return launch_convert_in<R>(c->st, n, (const double2*)in, c->Ta); }))) return s;
  } else {
    for (size_t off = 0; off < n; off += c->stage_elems) {
      const size_t mm = std::min(c->stage_elems, n - off);
      if ((s = c->cuda(cudaMemcpyAsync(c->stage, (const double2*)in + off, mm * sizeof(double2), cudaMemcpyHostToDevice, c->st), "apply_h stage"))) return s;
      if ((s = c->launch(KC_OTHER, "convert in", [&] { return launch_convert_in<R>(c->st, mm, c->stage, (float2*)c->Ta + off); }))) return s;
    }
  }
  if ((s = kinetic<R>(c, c->Ta, c->tmp, A))) return s;
  if ((s = gather<R>(c, c->Ta, A))) return s;
  if ((s = nl_scatter<R>(c, A))) return s;
  EpiParams ep{};
  ep.mode = EPI_APPLY;
  ep.nstates = c->nb;
  fill_shifts(c, A, ep.shift);
  ProjTables<R> pt = epi_tables<R>(c);
  const R* Vr = vsel<R>(c, true);
  if ((s = c->launch(KC_EPI, "apply H", [&] {
         return epilogue<R>(c, c->tmp, c->Ta, nullptr, c->Tb, nullptr, nullptr, Vr, pt, c->dcbuf, c->nkb, ep);
       })))
    return s;
  if (c->prec == TDDFT_FP64) {
    if ((s = c->cuda(cudaMemcpyAsync(out, c->Tb, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st), "apply_h out"))) return s;
  } else if (on_device) {
    if ((s = c->launch(KC_OTHER, "convert out", [&] { return launch_convert_out<R>(c->st, n, c->Tb, (double2*)out); }))) return s;
  } else {
    for (size_t off = 0; off < n; off += c->stage_elems) {
      const size_t mm = std::min(c->stage_elems, n - off);
      if ((s = c->launch(KC_OTHER, "convert out", [&] { return launch_convert_out<R>(c->st, mm, (const float2*)c->Tb + off, c->stage); }))) return s;
      if ((s = c->cuda(cudaMemcpyAsync((double2*)out + off, c->stage, mm * sizeof(double2), cudaMemcpyDeviceToHost, c->st), "apply_h stage out"))) return s;
      if ((s = c->cuda(cudaStreamSynchronize(c->st), "apply_h sync"))) return s;
    }
  }
  return c->cuda(cudaStreamSynchronize(c->st), "apply_h sync");
}

tddft_status create_impl(tddft_ctx* c, const tddft_cell* cell, const tddft_grid* grid, const tddft_atoms* atoms,
                         const tddft_projectors* pj, const tddft_params* pr) {
  if (!cell || !grid || !atoms || !pj || !pr) return c->fail(TDDFT_ERR_ARG, "null argument");
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j && cell->a[i][j] != 0.0) return c->fail(TDDFT_ERR_UNSUPPORTED, "only orthorhombic cells are supported");
  for (int i = 0; i < 3; ++i) {
    c->L[i] = cell->a[i][i];
    if (!(c->L[i] > 0.0)) return c->fail(TDDFT_ERR_ARG, "cell lengths must be positive");
  }
  if (grid->n[0] != grid->n[1] || grid->n[0] != grid->n[2]) return c->fail(TDDFT_ERR_UNSUPPORTED, "grid must be cubic (n x n x n)");
  if (!supported_n(grid->n[0])) return c->fail(TDDFT_ERR_UNSUPPORTED, "grid size must be one of 8, 12, 16, 24, 32, 48, 64, 96");
  c->N = grid->n[0];
  c->N3 = (size_t)c->N * c->N * c->N;
  c->omega = c->L[0] * c->L[1] * c->L[2];
  c->dV = c->omega / (double)c->N3;
  if (pr->precision != TDDFT_FP64 && pr->precision != TDDFT_FP32_MIXED) return c->fail(TDDFT_ERR_ARG, "bad precision");
  c->prec = pr->precision;
  c->proj_mode = pr->proj_mode;
  if (c->proj_mode < TDDFT_PROJ_FP64 || c->proj_mode > TDDFT_PROJ_F16X3) return c->fail(TDDFT_ERR_ARG, "bad proj_mode");
  if (pr->nk < 1 || pr->nk > kMaxK || !pr->kpts || !pr->kw) return c->fail(TDDFT_ERR_ARG, "nk must be 1..16 with kpts and kw");
  if (pr->nstates < 1 || !pr->occ) return c->fail(TDDFT_ERR_ARG, "nstates must be >= 1 with occ");
  c->nk = pr->nk;
  c->nb = pr->nstates;
  c->nkb = c->nk * c->nb;
  if (2 * c->nkb > 65535) return c->fail(TDDFT_ERR_UNSUPPORTED, "too many spinors (2 nk nstates must be <= 65535)");
  c->kpts.assign(pr->kpts, pr->kpts + 3 * c->nk);
  c->kw.assign(pr->kw, pr->kw + c->nk);
  c->occ.assign(pr->occ, pr->occ + c->nkb);
  c->wf.resize(c->nkb);
  for (int k = 0; k < c->nk; ++k)
    for (int b = 0; b < c->nb; ++b) c->wf[k * c->nb + b] = c->kw[k] * c->occ[k * c->nb + b];
  if (!(pr->dt != 0.0) || !std::isfinite(pr->dt)) return c->fail(TDDFT_ERR_ARG, "dt must be finite and non-zero");
  c->dt = pr->dt;
  if (pr->exp_kind != TDDFT_EXP_CHEBYSHEV && pr->exp_kind != TDDFT_EXP_TAYLOR && pr->exp_kind != TDDFT_EXP_CRANK_NICOLSON)
    return c->fail(TDDFT_ERR_ARG, "bad exp_kind");
  c->exp_kind = pr->exp_kind;
  c->exp_order = std::max(0, pr->exp_order);
  c->cheb_tol = pr->cheb_tol;
  c->n_sc = std::max(0, pr->n_sc);
  c->sc_tol = pr->sc_tol;
  c->emin_user = pr->e_min;
  c->emax_user = pr->e_max;
  if ((c->emin_user != 0.0 || c->emax_user != 0.0) && !(c->emax_user > c->emin_user))
    return c->fail(TDDFT_ERR_ARG, "e_max must exceed e_min");
  c->xc = pr->xc ? 1 : 0;
  {
    // TDDFT_NO_OVERLAP=1 keeps the gather on the main stream (same work, serial order)
    const char* e = std::getenv("TDDFT_NO_OVERLAP");
    if (!(e && e[0] == '1') &&
        (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      c->side = nullptr;
    }
  }
  c->spin_mode = pr->spin_mode;
  if (c->spin_mode < TDDFT_SPIN_NONCOLLINEAR || c->spin_mode > TDDFT_SPIN_UNPOLARISED)
    return c->fail(TDDFT_ERR_ARG, "spin_mode must be 0 (non-collinear), 1 (collinear) or 2 (unpolarised)");
  if (c->spin_mode != TDDFT_SPIN_NONCOLLINEAR && pj->lambda_so)
    for (int i = 0; i < pj->nspecies * (pj->lmax + 1); ++i)
      if (pj->lambda_so[i] != 0.0)
        return c->fail(TDDFT_ERR_ARG, "spin-orbit coupling couples the spin channels: it needs the non-collinear mode");
  {
    // FP32 xy passes take their planes through bulk asynchronous copies; TDDFT_NO_TMA=1 keeps
    // the register-fed passes (same results).
    const char* g = std::getenv("TDDFT_NO_TMA");
    c->use_tma = !(g && g[0] == '1');
    // The epilogue gives each thread one grid point of two spinors (with an even number of
    // states), so the projector scatter walks each point's entries once per spinor pair;
    // TDDFT_NO_EPI_PAIRS=1 keeps two points of one spinor per thread (same results).
    const char* h = std::getenv("TDDFT_NO_EPI_PAIRS");
    c->epi_pairs = !(h && h[0] == '1');
    // With the tensor-core projectors the Chebyshev epilogue runs inside the scatter kernel, so
    // V_NL psi never crosses HBM; TDDFT_NO_EPI_FUSE=1 keeps the scatter and the pointwise
    // epilogue apart (same arithmetic).
    const char* f = std::getenv("TDDFT_NO_EPI_FUSE");
    c->epi_fuse = !(f && f[0] == '1');
  }
  if (atoms->natoms < 0 || (atoms->natoms > 0 && (!atoms->pos || !atoms->species))) return c->fail(TDDFT_ERR_ARG, "bad atoms");
  c->natoms = atoms->natoms;
  if (c->natoms > 0) {
    if (pj->nspecies < 1 || !pj->Z || !pj->rc_loc || !pj->width || !pj->D || !pj->lambda_so) return c->fail(TDDFT_ERR_ARG, "bad projectors");
    if (pj->lmax < 0 || pj->lmax > 2) return c->fail(TDDFT_ERR_UNSUPPORTED, "lmax must be 0..2");
    if (!(pj->r_cut > 0.0) || pj->r_cut > 0.5 * std::min(c->L[0], std::min(c->L[1], c->L[2])))
      return c->fail(TDDFT_ERR_ARG, "r_cut must be positive and at most half the shortest cell side");
    for (int a = 0; a < c->natoms; ++a)
      if (atoms->species[a] < 0 || atoms->species[a] >= pj->nspecies) return c->fail(TDDFT_ERR_ARG, "species index out of range");
  }
  c->lmax = c->natoms > 0 ? pj->lmax : 0;
  c->nlm = (c->lmax + 1) * (c->lmax + 1);
  if (c->proj_mode >= TDDFT_PROJ_TF32 && c->prec == TDDFT_FP64)
    return c->fail(TDDFT_ERR_UNSUPPORTED, "tensor-core projectors need FP32-mixed precision");
  c->tile = c->proj_mode >= TDDFT_PROJ_TF32 && c->natoms > 0;
  if (c->tile && c->N % 16 != 0)
    return c->fail(TDDFT_ERR_UNSUPPORTED, "tensor-core projectors need a grid size divisible by 16");
  c->r_cut = pj->r_cut;
  c->pos.assign(atoms->pos, atoms->pos + 3 * c->natoms);
  std::vector<double> Zr(2 * std::max(1, c->natoms), 0.0);
  for (int a = 0; a < c->natoms; ++a) {
    Zr[2 * a] = pj->Z[atoms->species[a]];
    Zr[2 * a + 1] = pj->rc_loc[atoms->species[a]];
  }

  // ---- device allocations
  const size_t rs = c->rsize();
  const size_t pbytes = c->psi_elems() * 2 * rs;
  tddft_status s;
  if ((s = c->alloc(&c->psi, pbytes, "psi")) || (s = c->alloc(&c->phi, pbytes, "phi")) ||
      (s = c->alloc(&c->pred, pbytes, "pred")) || (s = c->alloc(&c->Ta, pbytes, "Ta")) ||
      (s = c->alloc(&c->Tb, pbytes, "Tb")) || (s = c->alloc(&c->tmp, pbytes, "tmp")))
    return s;
  const size_t ncoef = (size_t)c->nkb * std::max(1, c->natoms) * 2 * c->nlm;
  if ((s = c->alloc(&c->cbuf, ncoef * 2 * rs, "c")) || (s = c->alloc(&c->dcbuf, ncoef * 2 * rs, "dc"))) return s;
  const size_t N3 = c->N3;
  if ((s = c->alloc(&c->rho, 4 * N3 * 8, "rho")) || (s = c->alloc(&c->rho2, 4 * N3 * 8, "rho2")) ||
      (s = c->alloc(&c->rho3, 4 * N3 * 8, "rho3")) || (s = c->alloc(&c->V, 4 * N3 * 8, "V")) ||
      (s = c->alloc(&c->Vnew, 4 * N3 * 8, "Vnew")) || (s = c->alloc(&c->vloc, N3 * 8, "vloc")) ||
      (s = c->alloc(&c->vH, N3 * 8, "vH")) || (s = c->alloc(&c->exc, N3 * 8, "exc")) ||
      (s = c->alloc(&c->vxc4, 4 * N3 * 8, "vxc4")) || (s = c->alloc(&c->hart, N3 * 16, "hartree")) ||
      (s = c->alloc(&c->red, (16 + 5 * (size_t)c->nkb) * 8, "reductions")) || (s = c->alloc(&c->flag, 16, "flag")))
    return s;
  if (c->prec != TDDFT_FP64) {
    if ((s = c->alloc(&c->Vf, 4 * N3 * 4, "Vf")) || (s = c->alloc(&c->Vnewf, 4 * N3 * 4, "Vnewf"))) return s;
    c->stage_elems = std::min(c->psi_elems(), (size_t)(64u << 20) / sizeof(double2));
    if ((s = c->alloc(&c->stage, c->stage_elems * sizeof(double2), "stage"))) return s;
  }
  if ((s = upload(c, &c->wf_d, c->wf, "weights"))) return s;
  if (density_groups(N3, c->nkb) > 1 &&
      (s = c->alloc(&c->rho_part, (size_t)density_groups(N3, c->nkb) * 4 * N3 * 8, "density partials")))
    return s;
  if ((s = c->alloc(&c->tc_err, 16, "tc flag")) || (s = c->cuda(cudaMemset(c->tc_err, 0, 16), "tc flag init"))) return s;
  if ((s = c->cuda(cudaMemset(c->flag, 0, 16), "flag init"))) return s;

  // ---- twiddles exp(-2 pi i t / N)
  std::vector<double> tw(2 * c->N);
  for (int t = 0; t < c->N; ++t) {
    const long double ang = -2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)c->N;
    tw[2 * t] = (double)std::cos(ang);
    tw[2 * t + 1] = (double)std::sin(ang);
  }
  if ((s = upload(c, &c->tw64, std::vector<double2>((const double2*)tw.data(), (const double2*)tw.data() + c->N), "tw64")))
    return s;
  if (c->prec == TDDFT_FP64) {
    c->tw = c->tw64;
  } else if ((s = upload_typed<float>(c, &c->tw, tw, "tw32"))) {
    return s;
  }

  // ---- local potential on the device
  double* pos_d = nullptr;
  double* zr_d = nullptr;
  if ((s = upload(c, &pos_d, c->pos.empty() ? std::vector<double>(3, 0.0) : c->pos, "pos")) || (s = upload(c, &zr_d, Zr, "Zr")))
    return s;
  if ((s = c->alloc(&c->tq, (3 * (size_t)c->nkb + 8) * sizeof(double), "torque sums"))) return s;
  if ((s = c->alloc(&c->red_part, std::max(band_dot_part_doubles(c->nkb), field_sums_part_doubles()) * sizeof(double),
                    "reduction partials")))
    return s;
  if (c->natoms > 0) {
    if ((s = c->alloc(&c->owner, N3 * sizeof(int), "voronoi owner")) ||
        (s = c->alloc(&c->atom_sums, 4 * (size_t)c->natoms * 8, "atom sums")))
      return s;
    if ((s = c->launch(KC_OTHER, "voronoi owner", [&] {
           return launch_voronoi_owner(c->st, c->N, c->L, c->natoms, pos_d, c->owner);
         })))
      return s;
  }
  if ((s = c->launch(KC_OTHER, "vloc G", [&] { return launch_vloc_G(c->st, c->N, c->L, c->natoms, pos_d, zr_d, c->omega, c->hart); }))) return s;
  ZParams zp{};
  if ((s = c->launch(KC_OTHER, "vloc ifft z", [&] { return launch_fft_z<double>(c->st, c->N, c->hart, 1, c->tw64, Z_INV_ONLY, zp); }))) return s;
  if ((s = c->launch(KC_OTHER, "vloc ifft xy", [&] { return launch_fft_xy<double>(c->st, c->N, c->hart, c->hart, 1, c->tw64, true); }))) return s;
  if ((s = c->launch(KC_OTHER, "vloc real", [&] { return launch_complex_real_part(c->st, N3, c->hart, c->vloc, 1.0); }))) return s;

  // ---- projector tables
  HostTables ht;
  if (c->natoms > 0) {
    if ((s = build_tables(c, pj, atoms->species, ht))) return s;
    c->nl_bound = ht.nl_bound;
    c->n_entries = ht.g_idx.size();
    if ((s = upload(c, &c->g_ptr, ht.g_ptr, "g_ptr")) || (s = upload(c, &c->g_idx, ht.g_idx, "g_idx")) ||
        (s = upload(c, &c->s_ptr, ht.s_ptr, "s_ptr")) || (s = upload(c, &c->s_atom, ht.s_atom, "s_atom")))
      return s;
    {
      // spin-orbit torque matrices 2 i (D S_i - S_i D), S_i = sigma_i / 2 on the spin index of
      // the (projector, spin) index 2 p + sigma
      const int M = 2 * c->nlm;
      const cd sg[3][2][2] = {{{0.0, 1.0}, {1.0, 0.0}},
                              {{0.0, cd(0.0, -1.0)}, {cd(0.0, 1.0), 0.0}},
                              {{1.0, 0.0}, {0.0, -1.0}}};
      std::vector<double> T((size_t)c->natoms * 3 * M * M * 2, 0.0);
      for (int a = 0; a < c->natoms; ++a) {
        const double* Da = &ht.Dmat[(size_t)a * M * M * 2];
        auto D = [&](int r, int q) { return cd(Da[(r * M + q) * 2], Da[(r * M + q) * 2 + 1]); };
        for (int i = 0; i < 3; ++i)
          for (int r = 0; r < M; ++r)
            for (int q = 0; q < M; ++q) {
              // (D S)_{rq} = sum_s D_{r,(p_q,s)} S_{s,sigma_q};  (S D)_{rq} = sum_s S_{sigma_r,s} D_{(p_r,s),q}
              const int pq = q / 2, sq = q % 2, pr = r / 2, sr = r % 2;
              cd ds = 0.0, sd = 0.0;
              for (int s2 = 0; s2 < 2; ++s2) {
                ds += D(r, 2 * pq + s2) * 0.5 * sg[i][s2][sq];
                sd += 0.5 * sg[i][sr][s2] * D(2 * pr + s2, q);
              }
              const cd t = cd(0.0, 2.0) * (ds - sd);
              const size_t o = ((((size_t)a * 3 + i) * M + r) * M + q) * 2;
              T[o] = t.real();
              T[o + 1] = t.imag();
            }
      }
      double* Td = nullptr;
      if ((s = upload_typed<double>(c, reinterpret_cast<void**>(&Td), T, "soc torque"))) return s;
      c->Tsoc = reinterpret_cast<double2*>(Td);
    }
    // the full tables (d and the nlm projector values per entry) only feed the tensor-core
    // gather; the CUDA-core gather and the scatter evaluate beta from the compact rows
    if (c->prec == TDDFT_FP64) {
      if ((s = upload_typed<double>(c, &c->g_row, ht.g_row, "g_row")) || (s = upload_typed<double>(c, &c->s_row, ht.s_row, "s_row")) ||
          (s = upload_typed<double>(c, &c->nrm, ht.nrm, "nrm")) || (s = upload_typed<double>(c, &c->Dmat, ht.Dmat, "D")))
        return s;
    } else {
      if ((s = upload_typed<float>(c, &c->g_row, ht.g_row, "g_row")) || (s = upload_typed<float>(c, &c->s_row, ht.s_row, "s_row")) ||
          (s = upload_typed<float>(c, &c->nrm, ht.nrm, "nrm")) || (s = upload_typed<float>(c, &c->Dmat, ht.Dmat, "D")))
        return s;
    }
    if (c->tile) {
      const int ek = (c->proj_mode == TDDFT_PROJ_BF16X3) ? TILE_BF16 : (c->proj_mode == TDDFT_PROJ_F16X3) ? TILE_F16 : TILE_TF32;
      const int terms = (c->proj_mode == TDDFT_PROJ_TF32) ? 1 : 3;
      TileHost th;
      if ((s = build_tile_tables(c, ht, ek, terms, th))) return s;
      if (tile_scatter_smem(ek, terms, th.kch_max) > 227 * 1024)
        return c->fail(TDDFT_ERR_UNSUPPORTED, "too many projector spheres reach one brick for the tensor-core scatter");
      TileDev& td = c->td;
      td.ek = ek;
      td.terms = terms;
      td.BX = th.BX;
      td.nbx = th.nbx;
      td.nby = th.nby;
      td.nbz = th.nbz;
      td.nitems = (int)th.it_brick.size();
      td.natoms = c->natoms;
      td.nlm = c->nlm;
      td.smax = th.smax;
      td.kch_max = th.kch_max;
      for (int a = 0; a < 3; ++a) td.h[a] = c->L[a] / c->N;
      td.part_layer = (size_t)th.part_layer;
      int *ib, *ins, *inp, *ikc, *sa, *ap, *ai, *as;
      long long *igo, *iso, *ipo;
      float* sd;
      unsigned char *gt, *st2;
      if ((s = upload(c, &ib, th.it_brick, "tile bricks")) || (s = upload(c, &ins, th.it_nslot, "tile slots")) ||
          (s = upload(c, &inp, th.it_npad, "tile npad")) || (s = upload(c, &ikc, th.it_kch, "tile kch")) ||
          (s = upload(c, &igo, th.it_goff, "tile goff")) || (s = upload(c, &iso, th.it_soff, "tile soff")) ||
          (s = upload(c, &ipo, th.it_poff, "tile poff")) || (s = upload(c, &sa, th.slot_atom, "tile slot atoms")) ||
          (s = upload(c, &sd, th.slot_delta, "tile slot deltas")) || (s = upload(c, &gt, th.g_tab, "tile gather table")) ||
          (s = upload(c, &st2, th.s_tab, "tile scatter table")) || (s = upload(c, &ap, th.a_ptr, "tile atom ptr")) ||
          (s = upload(c, &ai, th.a_item, "tile atom items")) || (s = upload(c, &as, th.a_slot, "tile atom slots")))
        return s;
      td.it_brick = ib; td.it_nslot = ins; td.it_npad = inp; td.it_kch = ikc;
      td.it_goff = igo; td.it_soff = iso; td.it_poff = ipo;
      td.slot_atom = sa; td.slot_delta = reinterpret_cast<const float4*>(sd);
      td.g_tab = gt; td.s_tab = st2;
      td.a_ptr = ap; td.a_item = ai; td.a_slot = as;
      const size_t groups = (size_t)(2 * c->nb + 63) / 64;
      if ((s = c->alloc(&c->tile_part, (size_t)c->nk * groups * td.part_layer * sizeof(float) + 16, "tile partials")))
        return s;
      // points of bricks without projectors are never written by the scatter: zero once
      if ((s = c->alloc(&c->vnl, c->psi_elems() * 2 * sizeof(float), "vnl")) ||
          (s = c->cuda(cudaMemset(c->vnl, 0, c->psi_elems() * 2 * sizeof(float)), "vnl init")))
        return s;
    }
  }
  return c->cuda(cudaDeviceSynchronize(), "create sync");
}

}  // namespace

// =================================================================== C ABI

extern "C" {

tddft_status tddft_create(const tddft_cell* cell, const tddft_grid* grid, const tddft_atoms* atoms,
                          const tddft_projectors* proj, const tddft_params* params, tddft_handle* out) {
  if (!out) {
    g_create_error = "null output handle";
    return TDDFT_ERR_ARG;
  }
  *out = nullptr;
  tddft_ctx* c = new (std::nothrow) tddft_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return TDDFT_ERR_OOM;
  }
  tddft_status s = create_impl(c, cell, grid, atoms, proj, params);
  if (s != TDDFT_OK) {
    g_create_error = c->err;
    free_all(c);
    delete c;
    return s;
  }
  *out = c;
  return TDDFT_OK;
}

tddft_status tddft_set_fields(tddft_handle h, int nt, const double* t, const double* A, const double* B) {
  if (!h) return TDDFT_ERR_ARG;
  if (nt < 0 || (nt > 0 && (!t || !A || !B))) return h->fail(TDDFT_ERR_ARG, "bad field table");
  for (int i = 1; i < nt; ++i)
    if (!(t[i] > t[i - 1])) return h->fail(TDDFT_ERR_ARG, "field times must increase");
  h->ft.assign(t, t + nt);
  h->fA.assign(A, A + 3 * nt);
  h->fB.assign(B, B + 3 * nt);
  return TDDFT_OK;
}

tddft_status tddft_set_states(tddft_handle h, const void* psi, int on_device, double t0) {
  if (!h) return TDDFT_ERR_ARG;
  if (!psi) return h->fail(TDDFT_ERR_ARG, "null psi");
  return h->prec == TDDFT_FP64 ? do_set_states<double>(h, psi, on_device, t0) : do_set_states<float>(h, psi, on_device, t0);
}

tddft_status tddft_get_states(tddft_handle h, void* psi, int on_device) {
  if (!h) return TDDFT_ERR_ARG;
  if (!psi) return h->fail(TDDFT_ERR_ARG, "null psi");
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no states loaded");
  return h->prec == TDDFT_FP64 ? do_get_states<double>(h, psi, on_device) : do_get_states<float>(h, psi, on_device);
}

tddft_status tddft_set_states_c64(tddft_handle h, const void* psi, int on_device, double t0) {
  if (!h) return TDDFT_ERR_ARG;
  if (!psi) return h->fail(TDDFT_ERR_ARG, "null psi");
  return h->prec == TDDFT_FP64 ? do_set_states<double>(h, psi, on_device, t0, true)
                               : do_set_states<float>(h, psi, on_device, t0, true);
}

tddft_status tddft_get_states_c64(tddft_handle h, void* psi, int on_device) {
  if (!h) return TDDFT_ERR_ARG;
  if (!psi) return h->fail(TDDFT_ERR_ARG, "null psi");
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no states loaded");
  return store_states_c64(h, psi, on_device);
}

tddft_status tddft_step(tddft_handle h, int nsteps) {
  if (!h) return TDDFT_ERR_ARG;
  if (nsteps < 0) return h->fail(TDDFT_ERR_ARG, "nsteps must be >= 0");
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "tddft_set_states must come first");
  for (int i = 0; i < nsteps; ++i) {
    tddft_status s = h->prec == TDDFT_FP64 ? one_step<double>(h) : one_step<float>(h);
    if (s) return s;
  }
  return TDDFT_OK;
}

tddft_status tddft_observables(tddft_handle h, double* n, double* m, double* E, double* M, double* norms) {
  if (!h) return TDDFT_ERR_ARG;
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no states loaded");
  return h->prec == TDDFT_FP64 ? do_observables<double>(h, n, m, E, M, norms) : do_observables<float>(h, n, m, E, M, norms);
}

tddft_status tddft_get_potential(tddft_handle h, double* V) {
  if (!h || !V) return TDDFT_ERR_ARG;
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no states loaded");
  tddft_status s = h->cuda(cudaMemcpyAsync(V, h->V, 4 * h->N3 * sizeof(double), cudaMemcpyDeviceToHost, h->st), "potential read");
  if (s) return s;
  return h->cuda(cudaStreamSynchronize(h->st), "potential sync");
}

tddft_status tddft_apply_hamiltonian(tddft_handle h, const void* in, void* out, int on_device) {
  if (!h) return TDDFT_ERR_ARG;
  if (!in || !out || in == out) return h->fail(TDDFT_ERR_ARG, "bad in/out");
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no potential yet: call tddft_set_states first");
  return h->prec == TDDFT_FP64 ? do_apply_h<double>(h, in, out, on_device) : do_apply_h<float>(h, in, out, on_device);
}

tddft_status tddft_backward(tddft_handle h, int nsteps, int ckpt_every, const double* dL_drho, double* loss,
                            double* dL_dA, double* dL_dB) {
  if (!h) return TDDFT_ERR_ARG;
  if (nsteps < 1 || !dL_drho) return h->fail(TDDFT_ERR_ARG, "backward needs nsteps >= 1 and dL_drho");
  if (h->spin_mode != TDDFT_SPIN_NONCOLLINEAR)
    return h->fail(TDDFT_ERR_UNSUPPORTED, "the adjoint covers the non-collinear mode only");
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "tddft_set_states must come first");
  return h->prec == TDDFT_FP64 ? do_backward<double>(h, nsteps, ckpt_every, dL_drho, loss, dL_dA, dL_dB)
                               : do_backward<float>(h, nsteps, ckpt_every, dL_drho, loss, dL_dA, dL_dB);
}

tddft_status tddft_atom_moments(tddft_handle h, double* M, double* N) {
  if (!h) return TDDFT_ERR_ARG;
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no states loaded");
  if (h->natoms == 0) return TDDFT_OK;
  tddft_status s = h->launch(KC_OTHER, "atom sums", [&] {
    return launch_atom_sums(h->st, h->N3, h->natoms, h->rho, h->owner, h->atom_sums);
  });
  if (s) return s;
  std::vector<double> out(4 * (size_t)h->natoms);
  if ((s = h->cuda(cudaMemcpyAsync(out.data(), h->atom_sums, out.size() * 8, cudaMemcpyDeviceToHost, h->st), "atom read")) ||
      (s = h->cuda(cudaStreamSynchronize(h->st), "atom sync")))
    return s;
  for (int a = 0; a < h->natoms; ++a) {
    if (M)
      for (int c = 0; c < 3; ++c) M[3 * a + c] = out[4 * a + c] * h->dV;
    if (N) N[a] = out[4 * a + 3] * h->dV;
  }
  return TDDFT_OK;
}

tddft_status tddft_torques(tddft_handle h, double* soc, double* xc, double* zeeman) {
  if (!h) return TDDFT_ERR_ARG;
  if (!h->have_states) return h->fail(TDDFT_ERR_STATE, "no states loaded");
  double A[3], B[3];
  h->fields(h->t, A, B);
  tddft_status s;
  const int nkb = h->nkb;
  const bool nl = h->natoms > 0 && h->nlm > 0;
  if (nl) {
    // projections of the current states at k + A(t), then c^dagger 2 i [D, S] c per spinor
    if ((s = h->prec == TDDFT_FP64 ? gather<double>(h, h->psi, A) : gather<float>(h, h->psi, A))) return s;
    if ((s = h->launch(KC_OTHER, "soc torque", [&] {
           return h->prec == TDDFT_FP64
                      ? launch_soc_torque<double>(h->st, nkb, h->natoms, 2 * h->nlm, h->cbuf, h->Tsoc, h->tq)
                      : launch_soc_torque<float>(h->st, nkb, h->natoms, 2 * h->nlm, h->cbuf, h->Tsoc, h->tq);
         })))
      return s;
  }
  if ((s = h->launch(KC_OTHER, "xc torque", [&] { return launch_xc_torque(h->st, h->N3, h->rho, h->vxc4, h->tq + 3 * nkb); })))
    return s;
  std::vector<double> out(3 * (size_t)nkb + 6);
  if ((s = h->cuda(cudaMemcpyAsync(out.data(), h->tq, out.size() * 8, cudaMemcpyDeviceToHost, h->st), "torque read")) ||
      (s = h->cuda(cudaStreamSynchronize(h->st), "torque sync")))
    return s;
  double ts[3] = {0.0, 0.0, 0.0};
  if (nl)
    for (int kb = 0; kb < nkb; ++kb) {
      const double w = h->wf[kb];
      for (int i = 0; i < 3; ++i) ts[i] += w * out[3 * kb + i];
    }
  const double* f = out.data() + 3 * nkb;
  const double M[3] = {f[3] * h->dV, f[4] * h->dV, f[5] * h->dV};
  const double mu_b = 0.5;
  for (int i = 0; i < 3; ++i) {
    if (soc) soc[i] = ts[i];
    if (xc) xc[i] = 2.0 * f[i] * h->dV;
  }
  if (zeeman) {
    zeeman[0] = 2.0 * mu_b * (B[1] * M[2] - B[2] * M[1]);
    zeeman[1] = 2.0 * mu_b * (B[2] * M[0] - B[0] * M[2]);
    zeeman[2] = 2.0 * mu_b * (B[0] * M[1] - B[1] * M[0]);
  }
  return TDDFT_OK;
}

tddft_status tddft_set_wait_test_limit(unsigned first_polls) {
  using namespace tddft;
  const unsigned v = first_polls ? first_polls : (1u << 26);  // the kernels' default limit
  cudaError_t e = set_first_wait_fft(v);
  if (e == cudaSuccess) e = set_first_wait_tile(v);
  if (e != cudaSuccess) {
    set_global_error(std::string("tddft_set_wait_test_limit: ") + cudaGetErrorString(e));
    return TDDFT_ERR_CUDA;
  }
  return TDDFT_OK;
}

tddft_status tddft_set_stream(tddft_handle h, void* stream) {
  if (!h) return TDDFT_ERR_ARG;
  h->st = (cudaStream_t)stream;
  return TDDFT_OK;
}

tddft_status tddft_info(tddft_handle h, int* K_full, int* K_half, double* e_min, double* e_max, long long* launches) {
  if (!h) return TDDFT_ERR_ARG;
  if (K_full) *K_full = h->K_full;
  if (K_half) *K_half = h->K_half;
  if (e_min) *e_min = h->emin;
  if (e_max) *e_max = h->emax;
  if (launches) *launches = h->launches;
  return TDDFT_OK;
}

tddft_status tddft_profile(tddft_handle h, int enable) {
  if (!h) return TDDFT_ERR_ARG;
  tddft_status s = h->cuda(cudaStreamSynchronize(h->st), "profile sync");
  if (s) return s;
  for (auto& v : h->ev) v.clear();
  for (double& b : h->alg_bytes) b = 0.0;
  h->ev_used = 0;
  h->prof = enable != 0;
  return TDDFT_OK;
}

tddft_status tddft_profile_read(tddft_handle h, int ncls, double* ms, long long* count, double* bytes) {
  if (!h || ncls < 0 || ncls > kNumCls) return TDDFT_ERR_ARG;
  tddft_status s = h->cuda(cudaStreamSynchronize(h->st), "profile sync");
  if (s) return s;
  for (int c = 0; c < ncls; ++c) {
    double tot = 0.0;
    for (auto& e : h->ev[c]) {
      float x = 0.f;
      cudaEventElapsedTime(&x, e.first, e.second);
      tot += x;
    }
    if (ms) ms[c] = tot;
    if (count) count[c] = (long long)h->ev[c].size();
    if (bytes) bytes[c] = h->alg_bytes[c];
  }
  return TDDFT_OK;
}

const char* tddft_last_error(tddft_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

void tddft_destroy(tddft_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  free_all(h);
  delete h;
}

}  // extern "C"
