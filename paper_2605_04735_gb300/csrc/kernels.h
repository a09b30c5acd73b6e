// Host-side launchers of the library's kernels (one declaration per kernel
// family; definitions live in the .cu file of that family).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "common.cuh"
#include "modal.cuh"

namespace topo {

// ---- host helpers (topo.cu) ---------------------------------------------
// k0 (24x24, row-major) of the unit cube for E = 1 and Poisson ratio nu
void build_k0(double nu, double* k);

// ---- operator (operator.cu) -------------------------------------------
enum ApplyMode {
  APPLY_PLAIN = 0,  // y = A x
  APPLY_DOT = 1,    // y = A x, reduce x . y
  APPLY_RESID = 2   // y = f - A x (0 on fixed DOFs), reduce y . y
};
// errflag: set to 1 by the kernel if a bounded device-side wait ran out.
// mc != nullptr: element-centric modal kernel; nullptr: node-centric gather
// (one design only).  bt: designs of a mesh group (all pointers are design 0's).
template <typename T>
// energy (FP64 modal only, else nullptr): element energies
// (u_e - u_0)^T k0 (u_e - u_0) of x, written in the element layout.
cudaError_t launch_apply(const T* x, T* y, const T* E, const T* f, const Dims& d, const K0<T>& k0,
                         const ModalCoef<T>* mc, const Red& red, int mode, const int* done,
                         int* errflag, cudaStream_t s, const Bat& bt = Bat{},
                         T* energy = nullptr);
// The same operator (modal form) evaluated in double-word arithmetic (two
// FP32 words per value, ~48 significand bits): x given pre-split into hi and
// lo FP32 vectors (launch_split_dw), moduli E and f in FP64, y in FP64.
cudaError_t launch_apply_dw(const float* xh, const float* xl, double* y, const double* E,
                            const double* f, const Dims& d, const ModalCoef<double>& mc,
                            const Red& red, int mode, const int* done, cudaStream_t s,
                            const Bat& bt = Bat{});
// modal coefficients of k0 (returns false if k0 does not have the expected pattern)
bool build_modal_coef(const double* k0, ModalCoef<double>* out);
template <typename T>
cudaError_t launch_diag_inv(T* dinv, const T* E, const Dims& d, const K0<T>& k0, cudaStream_t s,
                            const Bat& bt = Bat{});

// ---- vectors (vectors.cu) -----------------------------------------------
// Every launcher takes the designs of a mesh group (default: one design).
// max_iter < 0: each design's max_iter_next
cudaError_t launch_set_max_iter(PcgScalars* sc, int max_iter, cudaStream_t s,
                                const Bat& bt = Bat{});
// n = total entries of one vector (3 * comp); all arrays 16-byte aligned
template <typename T>
cudaError_t launch_pcg_init(const T* b, T* x, T* r, T* z, T* p, const T* dinv, long long n,
                            const Red& red, bool jacobi, cudaStream_t s, const Bat& bt = Bat{});
// jacobi: z = D^-1 r and r.z; otherwise with dinv given z = D^-1 r scale
template <typename T>
cudaError_t launch_pcg_update(T* x, T* r, T* z, const T* p, const T* q, const T* dinv, long long n,
                              const Red& red, bool jacobi, cudaStream_t s, const Bat& bt = Bat{},
                              T scale = T(1));
template <typename T>
cudaError_t launch_pcg_direction(T* p, const T* z, long long n, const PcgScalars* sc,
                                 cudaStream_t s, const Bat& bt = Bat{});
template <typename T>
cudaError_t launch_dot(const T* a, const T* b, long long n, const Red& red, cudaStream_t s,
                       const Bat& bt = Bat{});
template <typename T>
cudaError_t launch_dot2(const T* a, const T* b, const T* c, long long n, const Red& red,
                        cudaStream_t s, const Bat& bt = Bat{});
// b32 = float(r64 * scale), scale = 1 / sqrt(sc->aux[0]) read on the device
// (batched launches skip the designs with sc->sat_out set, as does accumulate)
cudaError_t launch_narrow_scaled(float* b32, const double* r64, long long n, const PcgScalars* sc,
                                 cudaStream_t s, const Bat& bt = Bat{});
// u64 += scale * x, scale = sqrt(sc->aux[0]) read on the device (T = float or double)
template <typename T>
cudaError_t launch_accumulate(double* u64, const T* x, long long n, const PcgScalars* sc,
                              bool scaled, cudaStream_t s, const Bat& bt = Bat{});
template <typename T>
cudaError_t launch_copy_cast(T* dst, const double* src, long long n, cudaStream_t s,
                             const Bat& bt = Bat{});
// hi = float(u), lo = float(u - hi): the double-word split of an FP64 vector
// (skip: per-design flag, design-0 address; designs with it set are left alone)
cudaError_t launch_split_dw(const double* u, float* hi, float* lo, long long n, const int* skip,
                            cudaStream_t s, const Bat& bt = Bat{});

// ---- mesh data (meshdata.cu) -------------------------------------------
// rho (dense element order) -> ghosted rho32, E32, E64; counts bad values into *bad.
// Batched (bt): design b's input at b * src_stride floats from rho; rho_keep
// (optional) receives a copy of the input.
cudaError_t launch_simp(const float* rho, float* rho_g, float* E32, double* E64, const Dims& d,
                        double E0, double Emin, double penal, double hscale, int* bad,
                        cudaStream_t s, float* rho_keep = nullptr, long long src_stride = 0,
                        const Bat& bt = Bat{});
cudaError_t launch_build_load(double* f, const Dims& d, int load, double magnitude, double h,
                              cudaStream_t s);
// AoS (3n + c, dense node order) <-> ghosted SoA; unpack zeroes fixed DOFs
template <typename T>
cudaError_t launch_pack(const T* soa, double* aos, const Dims& d, cudaStream_t s);
template <typename T>
cudaError_t launch_unpack(const double* aos, T* soa, const Dims& d, cudaStream_t s);
// level-set stage (levelset.cu)
cudaError_t launch_shape_rhs(const double* u, const double* phi, double* part, double* bJ,
                             double* bV, const Dims& d, double eta, double E0, double nu,
                             double h, cudaStream_t s);
cudaError_t launch_hilb_setup(const double* f, uint8_t* dir, double* dinv, const Dims& d,
                              double ell2, double h, long long npad, cudaStream_t s);
cudaError_t launch_hilb_rhs(const double* src, double* b, const uint8_t* dir, const Dims& d,
                            long long npad, cudaStream_t s);
cudaError_t launch_hilb_apply(const double* x, double* y, const uint8_t* dir, const Dims& d,
                              double ell2, double h, const Red& red, bool dot, const int* done,
                              cudaStream_t s);
cudaError_t launch_hj_steps(double* phi, double* tmp, const double* v, const Dims& d,
                            double gamma, double h, int steps, unsigned long long* scratch,
                            double* dt_dev, cudaStream_t s);
cudaError_t launch_reinit_step(const double* phi, double* out, const Dims& d, double dt, double h,
                               unsigned long long* maxchange, cudaStream_t s);
// geometry transfer (transfer.cu)
cudaError_t launch_nodal_density(const float* rho, double* out, const Dims& d, double h,
                                 cudaStream_t s);
long long scan_scratch_count(long long n);
cudaError_t launch_mt_count(const double* f, long long* counts, long long* offsets,
                            long long* scratch, const Dims& d, double level, bool above, double h,
                            cudaStream_t s);
cudaError_t launch_mt_emit(const double* f, const long long* offsets, double* tris, const Dims& d,
                           double level, bool above, double h, cudaStream_t s);
cudaError_t launch_sdf(const double* tris, const long long* offsets, const double* rho_n,
                       double rho_t, double* phi, const Dims& d, double h, cudaStream_t s);
cudaError_t launch_ersatz(const double* phi, float* rho_g, float* E32, double* E64, const Dims& d,
                          double E0, double eta, double eps0, double hscale, const Red& red,
                          int* bad, cudaStream_t s);
// the same from stored element energies (the FP64 residual's by-product)
cudaError_t launch_sens_energy(const double* energy, const float* rho_g, const double* E64,
                               double* dc, const Dims& d, double penal, double dE, const Red& red,
                               cudaStream_t s, long long dc_stride = 0, const Bat& bt = Bat{});
// batched (bt): design b's output at b * dc_stride doubles from dc
cudaError_t launch_sensitivity(const double* u, const float* rho_g, const double* E64, double* dc,
                               const Dims& d, const ModalCoef<double>& kc, double penal, double dE,
                               const Red& red, cudaStream_t s, long long dc_stride = 0,
                               const Bat& bt = Bat{});

// ---- SIMP update (simp.cu) -------------------------------------------------
cudaError_t launch_filter(const double* dc, const float* rho_g, double* dcf, const Dims& d,
                          double radius, double guard, cudaStream_t s);
size_t oc_state_bytes();
size_t oc_partials_count();
cudaError_t launch_oc(const float* rho, const double* dcf, float* out, long long n, double volfrac,
                      double move, double eta, double rho_min, int passes, void* state,
                      double* partials, cudaStream_t s);
void oc_results(const void* state_host, double* sum, double* change, double* lambda);

}  // namespace topo
