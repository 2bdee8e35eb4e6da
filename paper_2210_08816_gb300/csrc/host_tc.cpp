// Host side of the tensor-core pressure-solve passes (FP32 operands of kernels_tc.cu, built in FP64):
// the mirror-symmetric half eigenproblems of every axis, the forward and backward matrices split into
// TF32 hi and FP32 lo parts, the eigenvalues in the tensor-core mode order, and the per-step B blocks in
// the shared-memory layout of the persistent pass.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "fv_internal.h"

namespace fv {

// B operands in the tensor-core order of the modes ([symmetric | antisymmetric], each by decreasing
// eigenvalue), built from the two half-size problems of the mirror-symmetric 1D operator: in the symmetric
// form B = W^-1/2 S W^-1/2 (tridiagonal d, e) the restriction to vectors with y[i] = +-y[n-1-i] is the
// leading (n/2) x (n/2) block with its last diagonal entry d[h-1] +- e[h-1] (the coupling across the
// midpoint).  Their eigenvectors, continued by mirror symmetry and scaled by 1/sqrt(2), are orthonormal
// eigenvectors of B that are exactly symmetric / antisymmetric (a full eigensolver returns arbitrary
// mixtures of the nearly degenerate wall-localised pairs of a stretched grid).  Per axis and direction
// two (h x h) matrices, each as TF32-exact hi and FP32 remainder:
//   forward  F_s[s][k] = sqrt(w_k / 2) y_s[k],   F_a[a][k] = sqrt(w_k / 2) y_a[k]     (k < h)
//   backward E_s[i][s] = y_s[i] / sqrt(2 w_i),   E_a[i][a] = y_a[i] / sqrt(2 w_i)     (i < h)
// plus the eigenvalues in that order.  Buffer: [axis][fwd_s_hi, fwd_s_lo, fwd_a_hi, fwd_a_lo, bwd_s_hi,
// bwd_s_lo, bwd_a_hi, bwd_a_lo][h x h], then [axis][lambda (n)], then the swizzled step blocks below.
int tc_host_operands(const int ns[3], const std::vector<double>* idx, const std::vector<double>* idc,
                     TcOperands& out) {
  std::vector<float>& hbuf = out.buf;
  size_t(&moff)[3][8] = out.moff;
  size_t(&loff)[3] = out.loff;
  size_t(&soff)[3][2] = out.soff;
  size_t total = 0;
  for (int d = 0; d < 3; ++d) total += 8 * (size_t)(ns[d] / 2) * (ns[d] / 2) + ns[d];
  const size_t sw_start = (total + 63) & ~(size_t)63;  // swizzled step blocks: 256-byte aligned
  total = sw_start;
  for (int d = 0; d < 3; ++d) total += 8 * (size_t)(ns[d] / 2) * (ns[d] / 2);
  hbuf.assign(total, 0.0f);
  size_t o = 0;
  auto put_split = [&](const std::vector<double>& M, size_t& ohi, size_t& olo, size_t cnt) {
    ohi = o;
    olo = o + cnt;
    for (size_t i = 0; i < cnt; ++i) {
      const float f = (float)M[i];
      uint32_t u;
      std::memcpy(&u, &f, 4);
      u = (u + 0x1000u) & 0xFFFFE000u;  // round to nearest TF32 (10 explicit mantissa bits)
      float hi;
      std::memcpy(&hi, &u, 4);
      hbuf[ohi + i] = hi;
      hbuf[olo + i] = (float)(M[i] - (double)hi);
    }
    o += 2 * cnt;
  };
  std::vector<double> lam_tc[3];
  for (int d = 0; d < 3; ++d) {
    const int n = ns[d], h = n / 2;
    std::vector<double> w(n), dg(n), off(n, 0.0);
    for (int i = 0; i < n; ++i) w[i] = 1.0 / idx[d][i];
    for (int i = 0; i < n; ++i) {
      double sdiag = 0.0;
      if (i >= 1) sdiag -= idc[d][i];
      if (i + 1 <= n - 1) sdiag -= idc[d][i + 1];
      dg[i] = sdiag / w[i];
      if (i + 1 <= n - 1) off[i] = idc[d][i + 1] / std::sqrt(w[i] * w[i + 1]);
    }
    std::vector<double> Ys, Ya, ls, la;
    for (int part = 0; part < 2; ++part) {
      std::vector<double> dd(dg.begin(), dg.begin() + h), ee(std::max(h - 1, 1), 0.0), Q;
      for (int i = 0; i + 1 < h; ++i) ee[i] = off[i];
      dd[h - 1] += (part == 0 ? 1.0 : -1.0) * off[h - 1];
      if (!tridiag_eig(h, dd, ee, Q)) return FV_EINVAL;
      std::vector<int> ord(h);
      for (int i = 0; i < h; ++i) ord[i] = i;
      std::sort(ord.begin(), ord.end(), [&](int a, int b) { return dd[a] > dd[b]; });
      std::vector<double> Y((size_t)h * h), L(h);
      for (int c = 0; c < h; ++c) {
        L[c] = dd[ord[c]];
        for (int i = 0; i < h; ++i) Y[(size_t)i * h + c] = Q[(size_t)i * h + ord[c]];
      }
      if (part == 0) {
        L[0] = 0.0;  // the constant vector: an exact null vector of the Neumann operator
        Ys = Y;
        ls = L;
      } else {
        Ya = Y;
        la = L;
      }
    }
    const size_t hh = (size_t)h * h;
    std::vector<double> Fs(hh), Fa(hh), Es(hh), Ea(hh);
    const double r2 = 1.0 / std::sqrt(2.0);
    for (int r = 0; r < h; ++r)
      for (int c = 0; c < h; ++c) {
        Fs[(size_t)r * h + c] = r2 * std::sqrt(w[c]) * Ys[(size_t)c * h + r];  // [mode r][cell c]
        Fa[(size_t)r * h + c] = r2 * std::sqrt(w[c]) * Ya[(size_t)c * h + r];
        Es[(size_t)r * h + c] = r2 * Ys[(size_t)r * h + c] / std::sqrt(w[r]);  // [cell r][mode c]
        Ea[(size_t)r * h + c] = r2 * Ya[(size_t)r * h + c] / std::sqrt(w[r]);
      }
    put_split(Fs, moff[d][0], moff[d][1], hh);
    put_split(Fa, moff[d][2], moff[d][3], hh);
    put_split(Es, moff[d][4], moff[d][5], hh);
    put_split(Ea, moff[d][6], moff[d][7], hh);
    lam_tc[d] = ls;
    lam_tc[d].insert(lam_tc[d].end(), la.begin(), la.end());
  }
  for (int d = 0; d < 3; ++d) {
    loff[d] = o;
    for (int m = 0; m < ns[d]; ++m) hbuf[o++] = (float)lam_tc[d][m];
  }
  // The persistent pass's B operands, per axis and direction: for every K step j the four slabs
  // [s_hi | s_lo | a_hi | a_lo] of rows 0..h-1 and columns 16 j .. 16 j + 15, each row's four 16-byte
  // chunks in the 64-byte swizzled order that a tensor-map copy into a 1024-byte aligned stage produces
  // (chunk c of row r at position c ^ ((r >> 1) & 3)), so that one contiguous bulk copy fills a stage.
  o = sw_start;
  for (int d = 0; d < 3; ++d) {
    const int h = ns[d] / 2, nstp = h / kTcSlabCols;
    for (int dir = 0; dir < 2; ++dir) {
      soff[d][dir] = o;
      for (int j = 0; j < nstp; ++j)
        for (int m = 0; m < 4; ++m) {
          const size_t src = moff[d][4 * dir + m];
          const size_t dst = o + (size_t)(j * 4 + m) * h * kTcSlabCols;
          for (int r = 0; r < h; ++r)
            for (int c = 0; c < 4; ++c) {
              const int pc = c ^ ((r >> 1) & 3);
              for (int e = 0; e < 4; ++e)
                hbuf[dst + (size_t)r * kTcSlabCols + pc * 4 + e] = hbuf[src + (size_t)r * h + j * kTcSlabCols + c * 4 + e];
            }
        }
      o += (size_t)nstp * 4 * h * kTcSlabCols;
    }
  }
  if (o != total) {
    set_error("tensor-core operand layout mismatch");
    return FV_EINVAL;
  }
  return FV_OK;
}

}  // namespace fv
