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
  clc::Buffer u[16], f[16], u0[16];  // per level: u with ghost ring, source, restricted u
  clc::Buffer coef[16];         // double[4][n] per level: aS, aN, b, area
  clc::Buffer invd[16];         // double[n][n] per level: 1 / diagonal
  clc::Buffer rot;              // double[npatch][9]: R_b (global -> patch frame)
  clc::Buffer coarse_inv;       // double[nc^2][nc^2]
  clc::Buffer psi_sht;          // double[12 nside_sht^2]
  clc::Buffer kappa_sht;        // double[12 nside_sht^2]
  clc::Buffer norms;            // double[npatch][2]
  clc::Buffer ratio;            // double[1]
  int cycles = 0;
  double residual = 0;
};

namespace clc {

struct MGView {
  int npatch;
  int n;           // finest cells per side
  double h;        // finest cell size
  const double* rot;
  const void* u;   // finest level potential with ghost ring
  int fp32;
};

MGView mg_view(const clc_plane_solution* sol);

}  // namespace clc
