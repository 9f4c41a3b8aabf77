// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/tddft.h"

namespace tddft {

constexpr int kMaxK = 16;      // k-points per handle
constexpr int kMaxNLM = 9;     // (lmax + 1)^2 with lmax <= 2
constexpr int kNumCls = 8;     // profiling classes

enum KernelClass { KC_FFT_XY = 0, KC_FFT_Z = 1, KC_EPI = 2, KC_PROJ = 3, KC_DENS = 4, KC_POT = 5, KC_OTHER = 6,
                   KC_SCATTER = 7 };

// Multiplier of the z pass: kinetic 1/2|G + s_k|^2 * scale, Poisson 4 pi / G^2 * scale.
struct ZParams {
  double gs[3];               // 2 pi / L_a
  double scale;
  int comps_per_k;            // spinor components per k-point (2 * nstates)
  double shift[kMaxK][3];     // k + A(t) per k-point
};

enum ZMode { Z_KIN = 0, Z_POISSON = 1, Z_INV_ONLY = 2 };

// Chebyshev / Taylor epilogue modes.
enum EpiMode { EPI_APPLY = 0, EPI_FIRST = 1, EPI_RECUR = 2, EPI_TAYLOR = 3, EPI_ADJ = 4, EPI_ADJ0 = 5 };

struct EpiParams {
  int mode;
  double c, inv_delta;          // H~ = (H - c) / Delta
  double a0[2], a1[2];          // accumulator 1 coefficients on T_k and T_{k+1}, complex
  double b0[2], b1[2];          // accumulator 2 coefficients
  double am[2], bm[2];          // unfused recurrence: coefficients on T_{k-1} (accumulators 1, 2)
  int use_acc1, use_acc2;
  int init1, init2;             // unfused recurrence: write the accumulator without reading it
  double shift[kMaxK][3];       // k + A(t), for projector phases
  int nstates;
  int dc_staged;                // fused kernel: D c copied to shared memory (set by its launcher)
  int spinor_pairs;             // epilogue: one point of two spinors per thread (even nstates)
  // FP32 kernels: c and 1 / Delta as {hi, lo}, the coefficients as {re hi, im hi, re lo, im lo}
  // (hi = the value rounded to float, lo = the rounded remainder; set by split_constants)
  float f_c[2], f_id[2];
  float f_a0[4], f_a1[4], f_b0[4], f_b1[4], f_am[4], f_bm[4];
};

// The series constants are applied identically at every term, every step and every grid point, so
// the rounding of one of them to FP32 is an error of the same sign everywhere: a coefficient off
// by a relative 6e-8 makes the propagator non-unitary by about that much per step, which adds up
// linearly over a run (and a rounded 1 / Delta rescales H).  FP32 kernels therefore apply each
// constant as the float pair hi + lo, exact to ~1e-14.
inline void split_constants(EpiParams& e) {
  auto s2 = [](double x, float* o) {
    o[0] = (float)x;
    o[1] = (float)(x - (double)o[0]);
  };
  auto s4 = [](const double* z, float* o) {
    o[0] = (float)z[0];
    o[1] = (float)z[1];
    o[2] = (float)(z[0] - (double)o[0]);
    o[3] = (float)(z[1] - (double)o[1]);
  };
  s2(e.c, e.f_c);
  s2(e.inv_delta, e.f_id);
  s4(e.a0, e.f_a0);
  s4(e.a1, e.f_a1);
  s4(e.b0, e.f_b0);
  s4(e.b1, e.f_b1);
  s4(e.am, e.f_am);
  s4(e.bm, e.f_bm);
}

// Device-side projector tables.
template <typename R> struct ProjTables {
  int natoms = 0, nlm = 0, ntab = 0;        // ntab = 3 + nlm reals per entry
  const int* g_ptr = nullptr;               // [natoms + 1] entries of each atom (gather order)
  const int* g_idx = nullptr;               // grid point of each gather entry
  const R* g_tab = nullptr;                 // [entries][3 + nlm]: d, beta
  const int* s_ptr = nullptr;               // [N^3 + 1] entries of each grid point (scatter order)
  const int* s_atom = nullptr;              // atom of each scatter entry
  const R* s_tab = nullptr;                 // [entries][3 + nlm]
  const R* Dmat = nullptr;                  // [natoms][2 nlm][2 nlm] complex (re, im)
  // Compact rows for the CUDA-core gather and the scatter: beta is evaluated from d as
  // N_l(w_a) g S_lm(d) with g = exp(-|d|^2 / (2 w_a^2)) and S_lm the real solid harmonics.
  const R* g_row = nullptr;                 // [entries][4]: d, g (gather order)
  const R* s_row = nullptr;                 // [entries][4] (scatter order)
  const R* nrm = nullptr;                   // [natoms][4]: N_0, N_1, N_2 of the atom's width, 0
  R yc[4] = {};                             // solid-harmonic constants: l = 0, l = 1, l = 2 (xy, ...), l = 2 (3z^2 - r^2)
};

// ---------------------------------------------------------------- launchers
template <typename R>
cudaError_t launch_fft_xy(cudaStream_t st, int N, const void* src, void* dst, int nbatch, const void* tw, bool inv);
// FP32 xy pass over persistent CTAs whose planes arrive by bulk asynchronous copies into
// double-buffered shared memory (two-factor sizes; src 16-byte aligned; src == dst allowed).
// err: bit 2 is set when a copy wait gave up.
bool fft_xy_tma_supported(int N);
cudaError_t launch_fft_xy_tma(cudaStream_t st, int N, const void* src, void* dst, int nbatch, const void* tw, bool inv,
                              int* err);
template <typename R>
cudaError_t launch_fft_z(cudaStream_t st, int N, void* data, int nbatch, const void* tw, int mode,
                         const ZParams& zp);
template <typename R>
cudaError_t launch_proj_gather(cudaStream_t st, int N, const void* psi, int nkb, const ProjTables<R>& pt,
                               double dV, const EpiParams& ep, void* c_out, void* dc_out);
template <typename R>
// kin: the kinetic part of H T_k; kin2 (may be null): V_NL T_k from the tensor-core scatter.
cudaError_t launch_epilogue(cudaStream_t st, int N, const void* kin, const void* kin2, const void* Tk,
                            const void* Tkm1, void* Tout, void* acc1, void* acc2, const R* V, const ProjTables<R>& pt,
                            const void* dc, int nkb, const EpiParams& ep);
// rho_v of all spinors; part (density_groups(N3, nkb) x 4 x N3 doubles, may be null) lets the
// band sum run as several groups reduced in a fixed order.
int density_groups(size_t N3, int nkb);
template <typename R>
cudaError_t launch_density(cudaStream_t st, size_t N3, const void* psi, int nkb, const double* wf,
                           double* rho, double* part);
cudaError_t launch_potential(cudaStream_t st, size_t N3, const double* rho, const double* vH,
                             const double* vloc, const double* B, int xc, int spin_mode, double* V, float* Vf,
                             double* exc, double* vxc4);
cudaError_t launch_density_to_complex(cudaStream_t st, size_t N3, const double* rho, double2* out);
cudaError_t launch_complex_real_part(cudaStream_t st, size_t N3, const double2* in, double* out, double scale);
cudaError_t launch_vloc_G(cudaStream_t st, int N, const double* L, int natoms, const double* pos,
                          const double* Zr, double omega, double2* out);
template <typename R>
cudaError_t launch_convert_in(cudaStream_t st, size_t n, const double2* in, void* out);
template <typename R>
cudaError_t launch_convert_out(cudaStream_t st, size_t n, const void* in, double2* out);
template <typename R>
cudaError_t launch_band_dot(cudaStream_t st, size_t npts, int nbands, const void* a, const void* b,
                            double* out2, double* part);  // part: band_dot_part_doubles(nbands)
size_t band_dot_part_doubles(int nbands);
template <typename R>
cudaError_t launch_nl_energy(cudaStream_t st, int nkb, int ncoef, const void* c, const void* dc, double* out);
cudaError_t launch_field_sums(cudaStream_t st, size_t N3, const double* rho, const double* vloc,
                              const double* vH, const double* exc, const double* vxc4, const double* V,
                              const double* B, double* out, double* part);  // part: field_sums_part_doubles()
size_t field_sums_part_doubles();
cudaError_t launch_max_abs_diff(cudaStream_t st, size_t n, const double* a, const double* b, double* out);
cudaError_t launch_check_window(cudaStream_t st, size_t N3, const double* V, double lo, double hi,
                                double kin_max, double nl_bound, int* flag);
// n and m (4 N3 doubles: n, m_x, m_y, m_z) from rho_v.
cudaError_t launch_nm_from_rho(cudaStream_t st, size_t N3, const double* rho, double* nm);
// min v, max v, max |b| of the potential (out3); part: field_sums_part_doubles() scratch.
cudaError_t launch_window_extrema(cudaStream_t st, size_t N3, const double* V, double* part, double* out3);

// ---------------------------------------------------------------- tile-centric tensor-core projectors
// Element kinds of the tensor-core operands.
enum { TILE_TF32 = 0, TILE_BF16 = 1, TILE_F16 = 2 };

// Device view of the brick tables (built at creation, see build_tile_tables in api.cu).  An
// "item" is a brick of BX x 8 x 8 points with at least one projector slot (atom image whose
// sphere reaches into the brick); items are in brick order.
struct TileDev {
  int ek = 0, terms = 1;                    // element kind, 1 or 3 (hi*hi + hi*lo + lo*hi) products
  int BX = 32, nbx = 0, nby = 0, nbz = 0;   // brick extent in x and bricks per axis
  int nitems = 0, natoms = 0, nlm = 0, smax = 0, kch_max = 0;
  double h[3] = {0, 0, 0};                  // grid spacing
  size_t part_layer = 0;                    // floats of partial products per (k-point, component group)
  const int* it_brick = nullptr;            // [nitems] linear brick index bx + nbx (by + nby bz)
  const int* it_nslot = nullptr;            // [nitems] slots
  const int* it_npad = nullptr;             // [nitems] gather N: nlm * nslot rounded up to 16
  const int* it_kch = nullptr;              // [nitems] scatter K chunks of 128 bytes
  const long long* it_goff = nullptr;       // [nitems] byte offset of the item's gather table
  const long long* it_soff = nullptr;       // [nitems] byte offset of the item's scatter table
  const long long* it_poff = nullptr;       // [nitems] float offset of the item's partial products
  const int* slot_atom = nullptr;           // [nitems][smax] atom of each slot
  const float4* slot_delta = nullptr;       // [nitems][smax] brick origin minus the atom image (bohr)
  const unsigned char* g_tab = nullptr;     // gather operand B: per item, chunk, part: npad rows x 128 B
  const unsigned char* s_tab = nullptr;     // scatter operand A: per item, tile, K chunk, part: 128 x 128 B
  const int* a_ptr = nullptr;               // [natoms + 1] (item, slot) pairs of each atom, in item order
  const int* a_item = nullptr;
  const int* a_slot = nullptr;
};
// Testing hook of the failure-detection path: polls of the first try of the bounded waits of the
// bulk-copy FFT pass and of the tensor-core gather (this device).
cudaError_t set_first_wait_fft(unsigned polls);
cudaError_t set_first_wait_tile(unsigned polls);
size_t tile_gather_smem(int terms);
size_t tile_scatter_smem(int ek, int terms, int kch_max);
// c[kb][a][2p + sigma] and dc = D c of every spinor (gather on the tensor cores, fixed-order
// reduction over the bricks); part: nk * groups * part_layer floats, groups = ceil(2 nstates / 64).
cudaError_t launch_tile_gather(cudaStream_t st, int N, const void* psi, int nk, int nstates, const TileDev& td,
                               double dV, const EpiParams& ep, const float* Dmat, float* part, void* c_out,
                               void* dc_out, int* err);
// Arrays of one Chebyshev term for the fused tensor-core epilogue (spinor layout; V the FP32
// potential 4-vector).
struct EpiIO {
  const float2* kin = nullptr;
  const float2* Tk = nullptr;
  const float2* Tkm1 = nullptr;
  float2* Tout = nullptr;
  float2* acc1 = nullptr;
  float2* acc2 = nullptr;
  const float* V = nullptr;
};
// The whole Chebyshev epilogue (modes EPI_FIRST, EPI_RECUR) of every point with V_NL from the
// tensor cores: one CTA per (component group, brick), every brick of the grid an item.
cudaError_t launch_tile_epilogue(cudaStream_t st, int N, int nk, int nstates, const TileDev& td, const EpiParams& ep,
                                 const void* dc, int* err, const EpiIO& io);
// out = V_NL psi from dc at the points of every brick with projectors (scatter on the tensor
// cores); out has the spinor layout and is left untouched elsewhere.
cudaError_t launch_tile_scatter(cudaStream_t st, int N, void* out, int nk, int nstates, const TileDev& td,
                                const EpiParams& ep, const void* dc, int* err);

// Voronoi (nearest-atom) cells and per-atom sums of m and n.
cudaError_t launch_voronoi_owner(cudaStream_t st, int N, const double* L, int natoms, const double* pos, int* owner);
// Spin-orbit torque per spinor: out[kb][i] = sum_a c_a^dagger T_a^i c_a (T: [natoms][3][M][M]
// complex FP64, M = 2 nlm); XC torque and magnetisation sums: out6 = {int b_xc x m, int m}
// without dV.
template <typename R>
cudaError_t launch_soc_torque(cudaStream_t st, int nkb, int natoms, int M, const void* c, const double2* T,
                              double* out);
cudaError_t launch_xc_torque(cudaStream_t st, size_t N3, const double* rho, const double* vxc4, double* out6);
cudaError_t launch_atom_sums(cudaStream_t st, size_t N3, int natoms, const double* rho, const int* owner, double* out);

// ---------------------------------------------------------------- adjoint launchers
template <typename R>
cudaError_t launch_grad_v(cudaStream_t st, size_t N3, int nkb, const void* S, const void* T, double f, double* gV,
                          double* part);  // part: density_groups(N3, nkb) x 4 N3 doubles
template <typename R>
cudaError_t launch_fft_z_current(cudaStream_t st, int N, void* U, const void* W, int nbatch, const void* tw,
                                 const ZParams& zp, double* part);
// Projector-phase A-gradient in one pass over the entries (replaces the moment gathers and
// launch_nl_agrad): out[kb][a] += f sum_atoms sum_e d_a Im(e^{-i phi}[conj(S) w_T + conj(T) w_S]).
// part: natoms x nkb x 3 doubles of scratch.
template <typename R>
cudaError_t launch_nl_agrad_fused(cudaStream_t st, int N, const void* S, const void* T, int nkb,
                                  const ProjTables<R>& pt, const EpiParams& ep, const void* dcS, const void* dcT,
                                  double f, double* part, double* out);
cudaError_t launch_xc_adjoint(cudaStream_t st, size_t N3, const double* rho, const double* gV, int xc, double* rbar,
                              double* gvf, double* gbf);
cudaError_t launch_add_hartree_adjoint(cudaStream_t st, size_t N3, const double2* h, double* rbar);
cudaError_t launch_real_field_to_complex(cudaStream_t st, size_t N3, const double* in, double2* out);
cudaError_t launch_sum3(cudaStream_t st, size_t N3, const double* g, double* out);
cudaError_t launch_accum_parts(cudaStream_t st, size_t count, const double* part, double f, double* out3);
template <typename R>
cudaError_t launch_density_adjoint(cudaStream_t st, size_t N3, int nkb, const void* psi, const double* rbar,
                                   const double* wf, const void* add, void* out);
template <typename R>
cudaError_t launch_seed(cudaStream_t st, size_t n, const void* y1, const double a[2], const void* y2,
                        const double b[2], void* out);

}  // namespace tddft
