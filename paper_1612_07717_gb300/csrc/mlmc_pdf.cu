// mlmc_pdf.cu -- the binned density of Section 6.3: per-level sums of the
// k smoothed bin QoIs (Eq. vector_QoI) and the adaptive MLMC estimate of the
// density, whose sample sizes use max_i Var[Y_{l,i}] in place of Var[Y_l]
// as the paper prescribes for the vector QoI.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "mlmc_internal.h"

namespace mlmc {


// Column sums of the per-block pdf partials, in block order (Kahan).
__global__ void __launch_bounds__(kBlock) k_finalize_pdf(const double* __restrict__ p, int nblocks,
                                                         int ncols, double* __restrict__ out) {
  const int col = blockIdx.x;
  __shared__ double s_w[kBlock / 32];
  double s = 0.0, c = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kBlock) {
    const double x = p[(size_t)b * ncols + col];
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  double v = s - c;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, ac = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) {
      const double y = s_w[w] - ac;
      const double t = a + y;
      ac = (t - a) - y;
      a = t;
    }
    out[col] = a - ac;
  }
}

static int pdf_grid(uint64_t N, int k) {
  DevInfo di;
  if (device_info(&di) != MLMC_OK) return 0;
  const size_t smem = (size_t)2 * k * kBlock * sizeof(double);
  int per_sm = (int)((200u * 1024u) / (smem > 0 ? smem : 1));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > kMaxBlocksPerSM) per_sm = kMaxBlocksPerSM;
  int g = di.sms * per_sm;
  const uint64_t need = (N + kBlock - 1) / kBlock;
  if (need < (uint64_t)g) g = (int)(need > 0 ? need : 1);
  return g;
}

}  // namespace mlmc

using namespace mlmc;

extern "C" {

int mlmc_level_pdf_sums(int level, uint64_t N, int integrator, const mlmc_params* p, uint64_t seed,
                        uint64_t path_offset, int k, void* workspace, size_t ws_bytes,
                        void* stream, double* out, uint64_t* n_ok, uint64_t* n_nonfinite) {
  if (!out || !n_ok || !n_nonfinite || k < 1 || k > kMaxPdfBins) return MLMC_EINVAL;
  if (integrator < MLMC_SE || integrator > MLMC_BAOAB || !p || !(p->smooth_delta > 0.0))
    return MLMC_EINVAL;
  HostModel hm;
  int rc = make_host_model(p, seed, &hm);
  if (rc) return rc;
  if (hm.adapt) return MLMC_EINVAL;  // the density kernel takes uniform timesteps
  LevelSpec ls;
  if ((rc = level_spec(hm, level, &ls))) return rc;
  if ((rc = check_stable(integrator, p, hm, ls))) return rc;
  Workspace w;
  if ((rc = carve(workspace, ws_bytes, &w))) return rc;
  const int grid = pdf_grid(N, k);
  if (grid <= 0) return MLMC_ENODEV;
  const int ncols = 2 * k + 2;
  double* partials = (double*)w.partials;
  double* res = (double*)w.results;
  cudaStream_t st = (cudaStream_t)stream;
  if (N > (uint64_t)grid * kBlock * 0x7FFFFFFFull) return MLMC_EINVAL;
  rc = cuda_status(launch_pdf(p->precision, integrator, hm, ls, N, path_offset, k, partials, grid, st));
  if (rc) return rc;
  k_finalize_pdf<<<ncols, kBlock, 0, st>>>(partials, grid, ncols, res);
  if ((rc = cuda_status(cudaGetLastError()))) return rc;
  double host[2 * kMaxPdfBins + 2];
  rc = cuda_status(cudaMemcpyAsync(host, res, ncols * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (!rc) rc = cuda_status(cudaStreamSynchronize(st));
  if (rc) return rc;
  std::memcpy(out, host, 2 * k * sizeof(double));
  *n_ok = (uint64_t)host[2 * k];
  *n_nonfinite = (uint64_t)host[2 * k + 1];
  return *n_nonfinite ? MLMC_ENONFINITE : MLMC_OK;
}

// Adaptive MLMC estimate of the binned density to RMSE eps per bin: the
// driver of mlmc_estimate with V_l = max_i Var[Y_{l,i}] (Section 6.3) and the
// bias test applied to every bin, max_i max(|Yhat_{L-1,i}| / 2, |Yhat_{L,i}|)
// < eps / sqrt(2).  pdf[i] = sum_l Yhat_{l,i}; out->estimate[0] is the total
// mass sum_i pdf[i], out->est_variance[0] the largest per-bin sum_l V_{l,i}/N_l,
// out->V[l] the largest per-bin variance of level l.
int mlmc_estimate_pdf(double eps, int integrator, const mlmc_params* p, uint64_t seed, int k,
                      void* workspace, size_t ws_bytes, void* stream, double* pdf,
                      mlmc_result* out) {
  if (!out || !pdf || !p || !(eps > 0.0) || k < 1 || k > kMaxPdfBins) return MLMC_EINVAL;
  if (p->L_max < p->level_min + 2 || p->L_max >= MLMC_MAX_LEVELS || p->n_init < 2)
    return MLMC_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<double> S((size_t)MLMC_MAX_LEVELS * 2 * k, 0.0);   // [l][2k]
  uint64_t n[MLMC_MAX_LEVELS] = {0}, bad[MLMC_MAX_LEVELS] = {0}, steps[MLMC_MAX_LEVELS] = {0};
  uint64_t Ndone[MLMC_MAX_LEVELS] = {0}, dN[MLMC_MAX_LEVELS] = {0};
  double V[MLMC_MAX_LEVELS] = {0}, C[MLMC_MAX_LEVELS] = {0};
  const int lmin = p->level_min;
  int L = lmin, converged = 0, status = MLMC_OK;
  auto var_of = [&](int l, int i) {
    const double nn = (double)n[l];
    const double m1 = S[(size_t)l * 2 * k + 2 * i], m2 = S[(size_t)l * 2 * k + 2 * i + 1];
    const double v = nn > 1.0 ? (m2 - m1 * m1 / nn) / (nn - 1.0) : 0.0;
    return v > 0.0 ? v : 0.0;
  };
  for (;;) {
    dN[L] = (uint64_t)p->n_init;
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = lmin; l <= L; ++l) {
        if (!dN[l]) continue;
        double sums[2 * kMaxPdfBins];
        uint64_t nok = 0, nbad = 0;
        int rc = mlmc_level_pdf_sums(l, dN[l], integrator, p, seed, Ndone[l], k, workspace,
                                     ws_bytes, stream, sums, &nok, &nbad);
        if (rc == MLMC_ENONFINITE) status = rc;
        else if (rc) return rc;
        for (int j = 0; j < 2 * k; ++j) S[(size_t)l * 2 * k + j] += sums[j];
        n[l] += nok;
        bad[l] += nbad;
        const int64_t M = (int64_t)p->M0 << l;
        steps[l] += dN[l] * (uint64_t)(l > lmin ? M + M / 2 : M);
        Ndone[l] += dN[l];
        dN[l] = 0;
      }
      if (pass == 1) break;
      double total = 0.0;
      for (int l = lmin; l <= L; ++l) {
        V[l] = 0.0;
        for (int i = 0; i < k; ++i) V[l] = std::fmax(V[l], var_of(l, i));
        const int64_t M = (int64_t)p->M0 << l;
        C[l] = l > lmin ? (double)(M + M / 2) : (double)M;
        total += std::sqrt(V[l] * C[l]);
      }
      for (int l = lmin; l <= L; ++l) {
        const double Nopt = std::ceil(2.0 / (eps * eps) * std::sqrt(V[l] / C[l]) * total);
        dN[l] = Nopt > (double)Ndone[l] ? (uint64_t)(Nopt - (double)Ndone[l]) : 0;
      }
    }
    if (L >= lmin + 2) {
      double rem = 0.0;
      for (int i = 0; i < k; ++i) {
        const double yL = std::fabs(S[(size_t)L * 2 * k + 2 * i] / (double)n[L]);
        const double yL1 = std::fabs(S[(size_t)(L - 1) * 2 * k + 2 * i] / (double)n[L - 1]);
        rem = std::fmax(rem, std::fmax(yL1 / 2.0, yL));
      }
      if (rem < eps / std::sqrt(2.0)) { converged = 1; break; }
    }
    if (L >= p->L_max) break;
    L += 1;
  }
  std::memset(out, 0, sizeof(*out));
  out->L = L;
  out->converged = converged;
  double mass = 0.0, worst = 0.0;
  for (int i = 0; i < k; ++i) {
    double est = 0.0, var = 0.0;
    for (int l = lmin; l <= L; ++l) {
      est += S[(size_t)l * 2 * k + 2 * i] / (double)n[l];
      var += var_of(l, i) / (double)n[l];
    }
    pdf[i] = est;
    mass += est;
    worst = std::fmax(worst, var);
  }
  out->estimate[0] = mass;
  out->est_variance[0] = worst;
  for (int l = lmin; l <= L; ++l) {
    out->N[l] = n[l];
    double vmax = 0.0, mmax = 0.0;
    for (int i = 0; i < k; ++i) {
      vmax = std::fmax(vmax, var_of(l, i));
      mmax = std::fmax(mmax, std::fabs(S[(size_t)l * 2 * k + 2 * i] / (double)n[l]));
    }
    out->V[l] = vmax;
    out->mean_y[l] = mmax;
    out->total_path_steps += steps[l];
    out->n_nonfinite += bad[l];
  }
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (status) return status;
  return converged ? MLMC_OK : MLMC_ENOTCONV;
}

}  // extern "C"
