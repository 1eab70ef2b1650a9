// brng_dirichlet.cuh -- Dirichlet rows and the LDA document-topic step: the
// per-unit body shared by brng_dirichlet.cu and the batched kernel.
//
// Sec. 1 (LDA paragraph and footnote): a K-dimensional Dirichlet deviate is
// K Gamma(alpha_k, 1) deviates y_k normalised by their sum.  Here each
// component k of a row-stream (a document) is its own Philox stream, so the
// K Gammas of a row are independent and run on different lanes: lane l of a
// warp owns components l, l+32, ... (P per lane, K <= 32 P).
//
// Rejection makes components finish a row at different times.  Instead of
// waiting at every row, a component may run up to `lookahead` (Q) rows ahead
// of the oldest row not yet normalised; finished log-Gammas wait in a
// per-warp shared queue q[Q][32P], and the warp normalises a row as soon as
// all components have produced it:
//     theta_k = exp(l_k - M) / sum_j exp(l_j - M),  M = max_j l_j,
// with l_k = log(d v) (+ log(u_b)/alpha_k when alpha_k < 1), which is
// y_k / sum y without underflow of tiny y_k.
//
// Bulk rows (brng_dirichlet): row-stream r serves rows r, r+R, r+2R, ... in
// order; a row whose alpha has an invalid entry is all NaN and consumes
// nothing (validity is voted by the warp for each row entering the window).
// LDA (brng_gibbs_run): the row is the document and every sweep redraws it
// with the same alpha; the warp accumulates theta in compensated (Kahan) FP32
// sums, added to the FP64 moments at the end (no FP64 instruction in the loop:
// GB300's FP64 pipe is narrow).
#pragma once

#include <cmath>

#include "brng_gamma.cuh"
#include "brng_internal.h"

namespace brng {

__host__ __device__ inline uint32_t dirichlet_warp_bytes(uint32_t P, uint32_t B, uint32_t Q) {
  return 128u + Q * 32u * P * 4u + 2u * P * B * 32u * 4u;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// One work unit (a row-stream of a bulk call, or a document), one warp;
// `base` holds dirichlet_warp_bytes(P, a.B, a.lookahead) bytes of shared memory.
template <int P, bool LDA>
__device__ __forceinline__ void dirichlet_unit(const DirichletArgs& a, uint64_t unit,
                                               unsigned char* base) {
  const unsigned lane = lane_id();
  const uint32_t Q = a.lookahead;
  const uint32_t KP = 32u * P;
  float* q = reinterpret_cast<float*>(base + 128);  // (the first 128 bytes are unused)
  float* rings = reinterpret_cast<float*>(base + 128 + Q * KP * 4u);
  const uint64_t n_units = LDA ? a.n_docs : (a.n_rows < a.R ? a.n_rows : a.R);
  if (unit >= n_units) return;  // whole warp
  const uint32_t K = a.K;
  const uint32_t nrows = LDA ? a.n_sweeps
                             : static_cast<uint32_t>((a.n_rows - unit + a.R - 1) / a.R);

  CRing<GenN> RN[P];
  CRing<GenU> RU[P];
  GammaState g[P];
  uint32_t stream[P], done[P];
  int att[P];
  bool kvalid[P], fresh[P];
  float acc32[P], comp32[P], last[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const uint32_t k = lane + 32u * p;
    kvalid[p] = k < K;
    const uint64_t sid = LDA ? (a.stream_base + unit) * K + k : unit * K + k;
    stream[p] = static_cast<uint32_t>(sid);
    uint64_t pn = 0, pu = 0;
    if (kvalid[p]) {
      if (LDA) {
        pn = a.pos[(unit * K + k) * 2];
        pu = a.pos[(unit * K + k) * 2 + 1];
      } else {
        pn = a.pos[static_cast<uint64_t>(a.S) + sid];
        pu = a.pos[sid];
      }
    }
    RN[p].init(rings + (2 * p) * a.B * 32u, nullptr, a.B, pn);
    RU[p].init(rings + (2 * p + 1) * a.B * 32u, nullptr, a.B, pu);
    done[p] = 0;
    att[p] = 0;
    fresh[p] = true;
    acc32[p] = 0.0f;
    comp32[p] = 0.0f;
    last[p] = 0.0f;
    g[p] = gamma_setup(1.0f);
  }

  // row validity over the window [tn, tn + Q): bit (row % Q)
  auto row_valid = [&](uint32_t m) -> bool {
    const uint64_t row = LDA ? unit : unit + static_cast<uint64_t>(m) * a.R;
    bool ok = true;
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (kvalid[p]) ok = ok && gamma_param_ok(a.alpha[row * K + lane + 32u * p]);
    return __all_sync(kFull, ok);
  };
  uint32_t vmask = 0;
  if (LDA) {
    const bool ok = row_valid(0);
    vmask = ok ? 0xffffffffu : 0u;
    count_warp(&a.cnt->n_domain, !ok && lane == 0);
  } else {
    for (uint32_t m = 0; m < Q && m < nrows; ++m) {
      const bool ok = row_valid(m);
      vmask |= (ok ? 1u : 0u) << m;
      count_warp(&a.cnt->n_domain, !ok && lane == 0);
    }
  }

  uint32_t tn = 0;
  while (tn < nrows) {
    bool run[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const bool work = kvalid[p] && done[p] < nrows && done[p] < tn + Q;
      const bool rowok = (vmask >> (done[p] % Q)) & 1u;
      if (work && !rowok) {  // invalid row: NaN, nothing consumed
        q[(done[p] % Q) * KP + lane + 32u * p] = __int_as_float(0x7fc00000);
        ++done[p];
        fresh[p] = true;
      }
      run[p] = work && rowok;
      if (run[p] && fresh[p]) {
        const uint64_t row = LDA ? unit : unit + static_cast<uint64_t>(done[p]) * a.R;
        g[p] = gamma_setup(a.alpha[row * K + lane + 32u * p]);
        fresh[p] = false;
      }
    }
    // one top-up point per ring: an attempt takes at most 1 N and 2 U (u, u_b)
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const bool live = kvalid[p] && done[p] < nrows;
      RN[p].ensure(run[p], 1, live, stream[p], a.rk);
      RU[p].ensure(run[p], 2, live, stream[p], a.rk);
    }
    // the P attempts of a lane are independent: no warp vote between them
    bool rejected = false, rechecked = false;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      float dv = 0.0f;
      float lb = 0.0f;  // log of the boost factor u_b^(1/alpha)
      bool rc = false;
      const bool acc = mt_attempt_peek<false, false, true>(run[p], g[p], RN[p], RU[p], stream[p], a.rk,
                                                           a.cnt, &dv, nullptr, &lb, &rc);
      rechecked = rechecked || rc;
      if (run[p]) {
        ++att[p];
        if (acc || att[p] >= kGammaMaxAttempts) {
          float l = __int_as_float(0x7fc00000);
          if (acc) {
            l = flog(dv) + lb;
          } else {
            rejected = true;
          }
          q[(done[p] % Q) * KP + lane + 32u * p] = l;
          ++done[p];
          att[p] = 0;
          fresh[p] = !LDA;
        }
      }
    }
    count_warp(&a.cnt->n_recheck, rechecked);
    count_warp(&a.cnt->n_reject, rejected);
    // normalise every row all components have finished
    uint32_t mn = 0xffffffffu;
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (kvalid[p]) mn = min(mn, done[p]);
    mn = __reduce_min_sync(kFull, mn);
    if (mn > nrows) mn = nrows;
    __syncwarp();
    while (tn < mn) {
      const uint32_t slot = tn % Q;
      float l[P];
      float M = -INFINITY;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        l[p] = kvalid[p] ? q[slot * KP + lane + 32u * p] : -INFINITY;
        M = fmaxf(M, l[p]);
      }
      M = warp_max(M);
      float e[P];
      float s = 0.0f;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        e[p] = kvalid[p] ? expf(l[p] - M) : 0.0f;
        s += e[p];
      }
      s = warp_sum(s);
      const float inv = 1.0f / s;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float th = e[p] * inv;
        if (LDA) {  // compensated (Kahan) FP32 sum: no FP64 in the loop
          const float yk = th - comp32[p];
          const float tk = acc32[p] + yk;
          comp32[p] = (tk - acc32[p]) - yk;
          acc32[p] = tk;
          last[p] = th;
        } else if (kvalid[p]) {
          const uint64_t row = unit + static_cast<uint64_t>(tn) * a.R;
          a.out[row * K + lane + 32u * p] = th;
        }
      }
      ++tn;
      if (!LDA && tn + Q - 1 < nrows) {
        const uint32_t m = tn + Q - 1;
        const bool ok = row_valid(m);
        vmask = (vmask & ~(1u << (m % Q))) | ((ok ? 1u : 0u) << (m % Q));
        count_warp(&a.cnt->n_domain, !ok && lane == 0);
      }
    }
    __syncwarp();
  }

  uint32_t left = 0;
#pragma unroll
  for (int p = 0; p < P; ++p)
    if (kvalid[p]) left += static_cast<uint32_t>(max(RN[p].avail(), 0) + max(RU[p].avail(), 0));
  count_waste(a.cnt, left);
#pragma unroll
  for (int p = 0; p < P; ++p) {
    if (!kvalid[p]) continue;
    const uint32_t k = lane + 32u * p;
    if (LDA) {
      const uint64_t idx = unit * K + k;
      a.pos[idx * 2] = RN[p].pos();
      a.pos[idx * 2 + 1] = RU[p].pos();
      a.out[idx] = last[p];
      a.moments[idx] += static_cast<double>(acc32[p]) - static_cast<double>(comp32[p]);
    } else {
      const uint64_t sid = unit * K + k;
      a.pos[static_cast<uint64_t>(a.S) + sid] = RN[p].pos();
      a.pos[sid] = RU[p].pos();
    }
  }
  __syncwarp();  // the rings are reused by the warp's next unit
}

}  // namespace brng
