// SHT+MG plane solver state (paper Sec. 3.2).
#pragma once

#include "common.cuh"

struct clc_plane_solution {
  clc_ctx* ctx = nullptr;
  int nside_fine = 0;
  clc_mg_params p{};
  int npatch = 0, nlev = 0;
  double h = 0;                 // finest cell size (radians)
  std::vector<int> sizes;       // cells per side per level
  clc::Buffer u[16], f[16];     // per level: correction e (colour-split rows, zero ghost ring), source
  clc::Buffer u2[16];           // per level but the coarsest: second correction buffer (pre-smoothed e)
  clc::Buffer base;             // double[npatch][(n+2)^2]: SHT solution inside, 2 g on the ring; final u
  clc::Buffer pvec;             // double[(n+2)^2][3]: patch-frame unit vectors of the finest level
  clc::Buffer ring_th_sht, ring_th_fine;  // ring colatitude tables
  clc::Buffer fnorm;            // double[npatch]: ||f||^2 of the source
  // interpolation plans (fixed by the patch geometry): 4 pixel indices and
  // weights per position, index -1 = position needs the 8-pixel pole stencil
  bool plan = false;
  clc::Buffer plan_psi_idx, plan_psi_w;   // [npatch][(n+2)^2]: int4, double[4]
  clc::Buffer plan_kap_idx, plan_kap_w;   // [npatch][n^2]
  // CLC_MIXED with plans: plan weights as float-float pairs, and float-float
  // copies of base, psi_SHT and kappa for the set-up on the FP32 pipe
  clc::Buffer base_ff, psi_ff, kap_ff;
  clc::Buffer coef[16];         // double[4][n] per level: aS, aN, b, area
  clc::Buffer invd[16];         // double[n][n] per level: 1 / diagonal
  clc::Buffer diag[16];         // double[n][n] per level: diagonal
  clc::Buffer rden[16];         // double[n/2] per level: 1 / (2 (area_2I + area_2I+1))
  clc::Buffer coef32[16], invd32[16], diag32[16], rden32[16];  // float copies
  clc::Buffer e64, e64b, fd64;  // CLC_MIXED: float-float correction, ping-pong (ghost-ring layout), defect source
  clc::Buffer coef_ff, diag_ff; // CLC_MIXED: finest-level operator coefficients as float-float pairs
  clc::Buffer rot;              // double[npatch][9]: R_b (global -> patch frame)
  clc::Buffer coarse_inv;       // double[nc^2][nc^2]
  clc::Buffer coarse_inv32;     // the same in FP32 (the FP32 V-cycles' coarsest solve)
  clc::Buffer psi_sht;          // double[12 nside_sht^2]
  clc::Buffer kappa_sht;        // double[12 nside_sht^2]
  clc::Buffer norms;            // double[npatch][2]
  clc::Buffer ratio;            // double[1]
  clc::Buffer wrow;             // double[n]: sin theta'_i of the finest rows (adjoint solve)
  clc::Buffer gc;               // double[npatch][4][n/2]: 2 psi_SHT at the coarse edge faces (tau rule)
  // partial sky (Sec. 3.4): patches only for a domain's bundles
  bool partial = false;
  clc::Buffer slot_bundle;      // int32[npatch]: NEST bundle of each patch slot
  clc::Buffer bundle_slot;      // int32[12 nside_bundle^2]: slot of each bundle, -1 outside the domain
  clc::Buffer outside;          // uint64: lookups outside the domain since the last solve
  clc::Buffer tau2;             // double[npatch]: ||tau||^2 over the coarse cells (tau rule)
  int cycles = 0;
  double residual = 0;
};

namespace clc {

struct MGView {
  int npatch;
  int n;           // finest cells per side
  double h;        // finest cell size
  double inv_h;    // 1 / h
  const double* rot;
  const double* u; // finest level potential u = u_SHT + e (ghost-ring layout)
  const int32_t* slot;           // bundle -> patch slot (NULL: slot = bundle); -1 outside the domain
  unsigned long long* outside;   // lookups of bundles outside the domain (partial sky)
};

MGView mg_view(const clc_plane_solution* sol);

// Adjoint of the converged SHT+MG patch solve of the plane held in `sol`
// (CLC_FP64 solutions): ubar[npatch][n][n] the adjoint of the finest interior
// potential; accumulates the transposed source interpolation into
// kbar_fine (RING map of nside_fine) and the transposed boundary-value
// interpolation into psibar_sht (RING map of nside_sht).  V-cycles until the
// max relative residual is below tol (or max_cycles).
int mg_adjoint_solve(clc_ctx* ctx, clc_plane_solution* s, const double* ubar, double tol, int max_cycles,
                     double* kbar_fine, double* psibar_sht, int* cycles_out, double* ratio_out);

}  // namespace clc
