// e+ e- -> mu+ mu- (QED, massless leptons): the one tree diagram, s-channel
// photon exchange (Feynman gauge), evaluated from the helicity spinors of all
// four leptons and the vector currents of the two fermion lines:
//   M(h) = e^2 [vbar(e+) gamma^mu u(e-)] [ubar(mu-) gamma_mu v(mu+)] / s
// up to a phase common to every helicity.  One thread per event loops over the
// 16 helicity configurations (each one costs two currents from the shared
// spinors and one Minkowski product), so the helicity sum needs no shuffles.
// The iteration reuses the sampling kernel and records of the other
// processes with massless final particles and a fixed partonic energy.
#include "mf_internal.h"
#include "mf_uux.cuh"

namespace mf {

// sum over the 16 helicities of |[vbar2 g^mu u1][ubar3 g_mu v4]|^2 / s^2
// (without MeParams::norm = e^4 / 4) for momenta in MadGraph order e-, e+, mu-, mu+
template <typename T> __device__ __forceinline__ T ee_me2(const T (&p)[4][4]) {
  R4<T> P[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) P[i].v[c] = p[i][c];
  R4<T> Q;
#pragma unroll
  for (int c = 0; c < 4; ++c) Q.v[c] = P[0].v[c] + P[1].v[c];
  const T s = mdot(Q, Q);
  V4<T> Le[2][2], Lm[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int la = 2 * a - 1;
    const S4<T> U1 = u_in(P[0], T(0), la), UB3 = ubar_out(P[2], T(0), la);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int lb = 2 * b - 1;
      Le[a][b] = vcur(vbar_in(P[1], T(0), lb), U1);
      Lm[a][b] = vcur(UB3, v_out(P[3], T(0), lb));
    }
  }
  T sum = T(0);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const cplx<T> m = mdot(Le[i >> 1][i & 1], Lm[j >> 1][j & 1]);
      sum = fma(m.r, m.r, fma(m.i, m.i, sum));
    }
  const T is = T(1) / s;
  return sum * is * is;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_matrix_element_ee(MeParams mp, int64_t n, const double* __restrict__ mom,
                                                                double* __restrict__ out) {
  for (int64_t e = int64_t(blockIdx.x) * kThreads + threadIdx.x; e < n; e += int64_t(gridDim.x) * kThreads) {
    T p[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[i][c] = T(mom[int64_t(i * 4 + c) * n + e]);
    out[e] = double(ee_me2<T>(p)) * mp.norm;
  }
}

// |M|^2 of the listed events (one thread each), weights, Vegas sums: the
// CTA's partial sums go to partials[blockIdx.x * nacc + k] as in k_me_acc
template <typename T>
__global__ void __launch_bounds__(kThreads) k_me_acc_ee(MeParams mp, int ndim, int nbins, RecordView<T> rec,
                                                        int accumulate, double* __restrict__ partials,
                                                        unsigned long long* __restrict__ counters,
                                                        double* __restrict__ w_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nacc = 2 + ndim * nbins;
  double* sums = reinterpret_cast<double*>(smem_raw);
  double* hist = sums + 2;
  const int t = threadIdx.x, lane = t & 31;
  for (int i = t; i < nacc; i += kThreads) sums[i] = 0.0;
  const unsigned full = 0xffffffffu;
  const int64_t npass = rec.count[0];
  double s1 = 0.0, s2 = 0.0;
  __syncthreads();
  for (int64_t k = int64_t(blockIdx.x) * kThreads + t; k < npass; k += int64_t(gridDim.x) * kThreads) {
    const int64_t e = rec.list[k];
    T p[4][4];
    const T rs = rec.rs[e];
    p[0][0] = T(0.5) * rs; p[0][1] = T(0); p[0][2] = T(0); p[0][3] = T(0.5) * rs;
    p[1][0] = T(0.5) * rs; p[1][1] = T(0); p[1][2] = T(0); p[1][3] = T(-0.5) * rs;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[2 + i][c] = rec.mom[int64_t(i * 4 + c) * rec.C + e];
    const double w = double(ee_me2<T>(p)) * mp.norm * rec.pref[e];
    s1 += w;
    s2 += w * w;
    if (w_out != nullptr) w_out[e] = w;
    for (int j = 0; j < ndim; ++j) atomicAdd(&hist[j * nbins + rec.flag[int64_t(j) * rec.C + e]], w * w);
  }
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(full, s1, off);
    s2 += __shfl_xor_sync(full, s2, off);
  }
  if (lane == 0) {
    atomicAdd(&sums[0], s1);
    atomicAdd(&sums[1], s2);
  }
  __syncthreads();
  double* dst = partials + int64_t(blockIdx.x) * nacc;
  for (int i = t; i < nacc; i += kThreads) dst[i] = (accumulate ? dst[i] : 0.0) + sums[i];
  if (t < 2) {
    const unsigned long long c = blockIdx.x == 0 ? (unsigned long long)rec.count[t] : 0ull;
    counters[blockIdx.x * 2 + t] = (accumulate ? counters[blockIdx.x * 2 + t] : 0ull) + c;
  }
}

namespace {
size_t ee_acc_smem(int ndim, int nbins) { return sizeof(double) * (2 + size_t(ndim) * nbins); }
}

cudaError_t ee_me_config(int precision, size_t* smem, int* ctas) {
  *smem = 0;
  if (precision == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_ee<double>, kThreads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_ee<float>, kThreads, 0);
}

cudaError_t ee_acc_config(int precision, int ndim, int nbins, size_t* smem, int* ctas) {
  *smem = ee_acc_smem(ndim, nbins);
  if (precision == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_ee<double>, kThreads, *smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_ee<float>, kThreads, *smem);
}

cudaError_t launch_matrix_element_ee(int precision, const MeParams& mp, int64_t n, const double* mom, double* out,
                                     int grid, cudaStream_t s) {
  if (precision == 0) k_matrix_element_ee<double><<<grid, kThreads, 0, s>>>(mp, n, mom, out);
  else k_matrix_element_ee<float><<<grid, kThreads, 0, s>>>(mp, n, mom, out);
  return cudaGetLastError();
}

cudaError_t launch_me_acc_ee(int precision, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                             int64_t C, int accumulate, double* partials, unsigned long long* counters, double* w_out,
                             int grid, cudaStream_t s) {
  const size_t sm = ee_acc_smem(ndim, nbins);
  if (precision == 0) {
    RecordView<double> rec = RecordView<double>::carve(rec_base, n_final, ndim, C);
    k_me_acc_ee<double><<<grid, kThreads, sm, s>>>(mp, ndim, nbins, rec, accumulate, partials, counters, w_out);
  } else {
    RecordView<float> rec = RecordView<float>::carve(rec_base, n_final, ndim, C);
    k_me_acc_ee<float><<<grid, kThreads, sm, s>>>(mp, ndim, nbins, rec, accumulate, partials, counters, w_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_chunk_ee(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                            int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                            int accumulate, double* partials, unsigned long long* counters, double* w_out, int grid,
                            cudaStream_t s, cudaEvent_t* ev) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + kThreads - 1) / kThreads;
  const int sgrid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);
  const size_t esm = sizeof(double) * sp.ndim * (sp.nbins + 1);
  cudaError_t e;
  if (precision == 0) {
    RecordView<double> rec = RecordView<double>::carve(rec_base, sp.n_final, sp.ndim, C);
    e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    k_sample_rec<double><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);
  } else {
    RecordView<float> rec = RecordView<float>::carve(rec_base, sp.n_final, sp.ndim, C);
    e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    k_sample_rec<float><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);
  }
  if (ev) cudaEventRecord(ev[1], s);
  e = launch_me_acc_ee(precision, mp, sp.n_final, sp.ndim, sp.nbins, rec_base, C, accumulate, partials, counters,
                       w_out, grid, s);
  if (ev) cudaEventRecord(ev[2], s);
  return e;
}

}  // namespace mf
