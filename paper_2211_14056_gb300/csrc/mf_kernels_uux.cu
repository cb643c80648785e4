// u u~ -> t t~ g g kernels: one event per warp, lane = helicities of
// (u, u~, t~, g, g) (bits 0..4), both top helicities per lane; the amplitude
// code is generated (mf_gen_uux.cuh).  The iteration reuses the sampling
// kernel and records of the gluon-initiated processes (same final state t t~
// g g, massless initial partons): k_me_acc_uux walks the list of events that
// passed, accumulates the weight and the Vegas sums like k_me_acc.
#include "mf_internal.h"
#include "mf_gen_uux.cuh"

namespace mf {

// The amplitude of one event (uux_config_me2, uux_warp_me2 below).
// p: physical momenta, p[0] beam 1 (+z), p[1] beam 2 (-z), p[2] t, p[3] tbar,
// p[4], p[5] the final light partons (a final gluon first).  The generated
// amplitude is that of u(P0) u~(P1) -> t(P2) t~(P3) g(P4) g(P5) with every
// momentum entering only through sums; the other subprocesses of p p -> t t~
// g g are its crossings, evaluated by filling its external slots (chan):
//   kChanQQB  u u~ -> t t~ g g        beams as they are
//   kChanQBQ  u~ u -> t t~ g g        the quark from beam 2
//   kChanQG   u g  -> t t~ g u        the u~ slot takes the outgoing quark,
//                                      ubar(p5) at momentum -p5; the first gluon
//                                      slot the incoming gluon, eps(p1) at -p1
//   kChanGQ   g u  -> t t~ g u        the same with the beams exchanged
//   kChanQBG  u~ g -> t t~ g u~       charge conjugate of u g -> t~ t g u: the
//   kChanGQB  g u~ -> t t~ g u~       quark slots take the antiquarks' momenta,
//                                      the top slots exchange t and t~
// (a crossed fermion flips the amplitude's sign, which |M|^2 does not see;
// the colour decomposition is over index slots and does not change).
// (the kChan* codes are declared beside MeParams)

// |M|^2 (without MeParams::norm) of one helicity configuration cfg of the
// amplitude's slots (bit 0: the incoming quark slot, 1: the light antifermion
// slot, 2: the antitop slot, 3 and 4: the two gluon slots; helicity +1 where
// set), both helicities of the top slot summed; every thread on its own.
template <typename T>
__device__ __forceinline__ T uux_config_me2(const T (&p)[6][4], T mt, T mw, int chan, unsigned cfg) {
  R4<T> Q[6];
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) Q[i].v[c] = p[i][c];
  const int l1 = (cfg & 1) ? 1 : -1, l2 = (cfg & 2) ? 1 : -1, l4 = (cfg & 4) ? 1 : -1;
  const int l5 = (cfg & 8) ? 1 : -1, l6 = (cfg & 16) ? 1 : -1;
  const bool swap_beams = chan == kChanQBQ || chan == kChanGQ || chan == kChanGQB;
  const bool crossed = chan >= kChanQG;
  const bool conj_tops = chan == kChanQBG || chan == kChanGQB;
  const R4<T>& qin = swap_beams ? Q[1] : Q[0];      // the incoming (anti)quark on the amplitude's quark line
  const R4<T>& other = swap_beams ? Q[0] : Q[1];    // the other beam parton
  const R4<T>& top = conj_tops ? Q[3] : Q[2];
  const R4<T>& atop = conj_tops ? Q[2] : Q[3];
  R4<T> P[6];
  P[0] = qin;
  P[2] = top;
  P[3] = atop;
  S4<T> V2;
  V4<T> E5, E6;
  if (crossed) {
    P[1] = -Q[5];
    P[4] = -other;
    P[5] = Q[4];
    V2 = ubar_out(Q[5], T(0), l2);
    E5 = polarisation(other, l5, false);
    E6 = polarisation(Q[4], l6, true);
  } else {
    P[1] = other;
    P[4] = Q[4];
    P[5] = Q[5];
    V2 = vbar_in(other, T(0), l2);
    E5 = polarisation(Q[4], l5, true);
    E6 = polarisation(Q[5], l6, true);
  }
  const S4<T> U1 = u_in(qin, T(0), l1);
  const S4<T> VTB = v_out(atop, mt, l4);
  const S4<T> UB3[2] = {ubar_out(top, mt, -1), ubar_out(top, mt, 1)};
  cplx<T> J[2][kUuxFlows];
  uux_amplitudes<T>(P, mt, mw, U1, V2, VTB, UB3, E5, E6, J);
  return uux_colour_form<T>(J[0]) + uux_colour_form<T>(J[1]);
}

// The sum over the 32 configurations, lane = configuration; every lane of the
// warp calls it and receives the sum.
template <typename T>
__device__ __forceinline__ T uux_warp_me2(const T (&p)[6][4], T mt, T mw, int chan) {
  T part = uux_config_me2<T>(p, mt, mw, chan, unsigned(threadIdx.x & 31));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  return part;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_matrix_element_uux(MeParams mp, int64_t n, const double* __restrict__ mom,
                                                                 double* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T mt = T(mp.mt), mw = T(mp.mw);
  for (int64_t e = int64_t(blockIdx.x) * kWarps + warp; e < n; e += int64_t(gridDim.x) * kWarps) {
    T p[6][4];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[i][c] = T(mom[int64_t(i * 4 + c) * n + e]);
    const T v = uux_warp_me2<T>(p, mt, mw, mp.chan);
    if (lane == 0) out[e] = double(v) * mp.norm;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_me_acc_uux(MeParams mp, int ndim, int nbins, RecordView<T> rec,
                                                         int accumulate, double* __restrict__ partials,
                                                         unsigned long long* __restrict__ counters,
                                                         double* __restrict__ w_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nacc = 2 + ndim * nbins;
  double* sums = reinterpret_cast<double*>(smem_raw);
  double* hist = sums + 2;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < nacc; i += kThreads) sums[i] = 0.0;
  const T mt = T(mp.mt), mw = T(mp.mw);
  const unsigned full = 0xffffffffu;
  const int64_t npass = rec.count[0];
  double s1 = 0.0, s2 = 0.0;
  __syncthreads();
  for (int64_t k = int64_t(blockIdx.x) * kWarps + warp; k < npass; k += int64_t(gridDim.x) * kWarps) {
    const int64_t e = rec.list[k];
    T p[6][4];
    const T rs = rec.rs[e];
    p[0][0] = T(0.5) * rs; p[0][1] = T(0); p[0][2] = T(0); p[0][3] = T(0.5) * rs;
    p[1][0] = T(0.5) * rs; p[1][1] = T(0); p[1][2] = T(0); p[1][3] = T(-0.5) * rs;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[2 + i][c] = rec.mom[int64_t(i * 4 + c) * rec.C + e];
    const T v = uux_warp_me2<T>(p, mt, mw, mp.chan);
    const double w = double(v) * mp.norm * rec.pref[e];
    if (lane == 0) {
      s1 += w;
      s2 += w * w;
      if (w_out != nullptr) w_out[e] = w;
    }
    if (lane < ndim) atomicAdd(&hist[lane * nbins + rec.flag[int64_t(lane) * rec.C + e]], w * w);
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

// ----------------------------------------------------------------------------
// Helicity sampling: one event per thread, its configuration given (hel) or
// drawn from the grid's thresholds (k_me_acc_uux_hel); the same per-thread
// amplitude code as the summing kernels, which give each lane one
// configuration of one event.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_matrix_element_uux_hel(MeParams mp, int64_t n,
                                                                     const double* __restrict__ mom,
                                                                     const int* __restrict__ hel,
                                                                     double* __restrict__ out) {
  const T mt = T(mp.mt), mw = T(mp.mw);
  for (int64_t e = int64_t(blockIdx.x) * kThreads + threadIdx.x; e < n; e += int64_t(gridDim.x) * kThreads) {
    T p[6][4];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) p[i][c] = T(mom[int64_t(i * 4 + c) * n + e]);
    out[e] = double(uux_config_me2<T>(p, mt, mw, mp.chan, unsigned(hel[e]) & 31u)) * mp.norm;
  }
}

// Shared memory of k_me_acc_uux_hel: Vegas sums, histogram, the draw's 33
// thresholds, the 32 configurations' sums of squared weights.
struct UuxHelLayout {
  __host__ __device__ static size_t al(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ static size_t thr(int nacc) { return al(sizeof(double) * nacc); }
  __host__ __device__ static size_t hsq(int nacc) { return al(thr(nacc) + sizeof(unsigned long long) * 33); }
  __host__ __device__ static size_t total(int nacc) { return al(hsq(nacc) + sizeof(double) * 32); }
};

// Weights w = |M_h|^2 norm * prefactor / p_h of the listed events, one thread
// per event, and the Vegas sums; with hel_sq given, the CTA's per-configuration
// sums of squared weights (as k_me_acc_hel).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_me_acc_uux_hel(MeParams mp, int ndim, int nbins, RecordView<T> rec,
                                                             int accumulate, double* __restrict__ partials,
                                                             unsigned long long* __restrict__ counters,
                                                             double* __restrict__ w_out, uint64_t seed, int iter,
                                                             int64_t first_event,
                                                             const unsigned long long* __restrict__ hel_T,
                                                             double* __restrict__ hel_sq) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nacc = 2 + ndim * nbins;
  double* sums = reinterpret_cast<double*>(smem_raw);
  double* hist = sums + 2;
  unsigned long long* thr = reinterpret_cast<unsigned long long*>(smem_raw + UuxHelLayout::thr(nacc));
  double* hsq = reinterpret_cast<double*>(smem_raw + UuxHelLayout::hsq(nacc));
  const int t = threadIdx.x;
  for (int i = t; i < nacc; i += kThreads) sums[i] = 0.0;
  if (t <= 32) thr[t] = hel_T[t];
  if (t < 32) hsq[t] = 0.0;
  const T mt = T(mp.mt), mw = T(mp.mw);
  const int64_t npass = rec.count[0];
  __syncthreads();
  // warp-uniform trip count: every lane takes part in the accumulation's shuffles
  for (int64_t base = int64_t(blockIdx.x) * kThreads + (t & ~31); base < npass;
       base += int64_t(gridDim.x) * kThreads) {
    const int64_t k = base + (t & 31);
    const bool ok = k < npass;
    double w = 0.0;
    uint8_t b_ev[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) b_ev[j] = 0;
    if (ok) {
      const int64_t e = rec.list[k];
      T p[6][4];
      const T rs = rec.rs[e];
      p[0][0] = T(0.5) * rs; p[0][1] = T(0); p[0][2] = T(0); p[0][3] = T(0.5) * rs;
      p[1][0] = T(0.5) * rs; p[1][1] = T(0); p[1][2] = T(0); p[1][3] = T(-0.5) * rs;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) p[2 + i][c] = rec.mom[int64_t(i * 4 + c) * rec.C + e];
      const unsigned h = helicity_draw<4>(helicity_word(seed, iter, uint64_t(first_event + e)), thr);
      const T v = uux_config_me2<T>(p, mt, mw, mp.chan, h);
      w = double(v) * mp.norm * rec.pref[e] * (4294967296.0 / double(thr[h + 1] - thr[h]));
      if (w_out != nullptr) w_out[e] = w;
      if (hel_sq != nullptr) atomicAdd(&hsq[h], w * w);
#pragma unroll
      for (int j = 0; j < kMaxDim; ++j)
        if (j < ndim) b_ev[j] = rec.flag[int64_t(j) * rec.C + e];
    }
    accumulate_event(w, b_ev, ndim, nbins, sums, hist);
  }
  __syncthreads();
  double* dst = partials + int64_t(blockIdx.x) * nacc;
  for (int i = t; i < nacc; i += kThreads) dst[i] = (accumulate ? dst[i] : 0.0) + sums[i];
  if (t < 2) {
    const unsigned long long c = blockIdx.x == 0 ? (unsigned long long)rec.count[t] : 0ull;
    counters[blockIdx.x * 2 + t] = (accumulate ? counters[blockIdx.x * 2 + t] : 0ull) + c;
  }
  if (hel_sq != nullptr && t < 32) {
    double* d = hel_sq + int64_t(blockIdx.x) * kHelMaxConfigs + t;
    *d = (accumulate ? *d : 0.0) + hsq[t];
  }
}

namespace {
size_t acc_smem(int ndim, int nbins) { return sizeof(double) * (2 + size_t(ndim) * nbins); }
}

cudaError_t uux_hel_me_config(int precision, int* ctas) {
  if (precision == 0)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_uux_hel<double>, kThreads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_uux_hel<float>, kThreads, 0);
}

cudaError_t uux_hel_acc_config(int precision, int ndim, int nbins, int* ctas) {
  const size_t sm = UuxHelLayout::total(2 + ndim * nbins);
  if (precision == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_uux_hel<double>, kThreads, sm);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_uux_hel<float>, kThreads, sm);
}

cudaError_t launch_matrix_element_uux_hel(int precision, const MeParams& mp, int64_t n, const double* mom,
                                          const int* hel, double* out, int grid, cudaStream_t s) {
  if (precision == 0) k_matrix_element_uux_hel<double><<<grid, kThreads, 0, s>>>(mp, n, mom, hel, out);
  else k_matrix_element_uux_hel<float><<<grid, kThreads, 0, s>>>(mp, n, mom, hel, out);
  return cudaGetLastError();
}

cudaError_t uux_me_config(int precision, size_t* smem, int* ctas) {
  *smem = 0;
  if (precision == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_uux<double>, kThreads, 0);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_matrix_element_uux<float>, kThreads, 0);
}

cudaError_t uux_acc_config(int precision, int ndim, int nbins, size_t* smem, int* ctas) {
  *smem = acc_smem(ndim, nbins);
  if (precision == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_uux<double>, kThreads, *smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_me_acc_uux<float>, kThreads, *smem);
}

cudaError_t launch_matrix_element_uux(int precision, const MeParams& mp, int64_t n, const double* mom, double* out,
                                      int grid, cudaStream_t s) {
  if (precision == 0) k_matrix_element_uux<double><<<grid, kThreads, 0, s>>>(mp, n, mom, out);
  else k_matrix_element_uux<float><<<grid, kThreads, 0, s>>>(mp, n, mom, out);
  return cudaGetLastError();
}

cudaError_t launch_me_acc_uux(int precision, const MeParams& mp, int n_final, int ndim, int nbins, void* rec_base,
                              int64_t C, int accumulate, double* partials, unsigned long long* counters,
                              double* w_out, int grid, cudaStream_t s) {
  const size_t sm = acc_smem(ndim, nbins);
  if (precision == 0) {
    RecordView<double> rec = RecordView<double>::carve(rec_base, n_final, ndim, C);
    k_me_acc_uux<double><<<grid, kThreads, sm, s>>>(mp, ndim, nbins, rec, accumulate, partials, counters, w_out);
  } else {
    RecordView<float> rec = RecordView<float>::carve(rec_base, n_final, ndim, C);
    k_me_acc_uux<float><<<grid, kThreads, sm, s>>>(mp, ndim, nbins, rec, accumulate, partials, counters, w_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_chunk_uux(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
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
  e = launch_me_acc_uux(precision, mp, sp.n_final, sp.ndim, sp.nbins, rec_base, C, accumulate, partials, counters,
                        w_out, grid, s);
  if (ev) cudaEventRecord(ev[2], s);
  return e;
}

cudaError_t launch_chunk_uux_hel(int precision, const SampleParams& sp, const MeParams& mp, const double* edges,
                                 int64_t first_event, int64_t n, int64_t C, void* rec_base, uint64_t seed, int iter,
                                 int accumulate, double* partials, unsigned long long* counters, double* w_out,
                                 int grid, cudaStream_t s, cudaEvent_t* ev, const unsigned long long* hel_T,
                                 double* hel_sq) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int64_t need = (n + kThreads - 1) / kThreads;
  const int sgrid = int(need < int64_t(sms) * 16 ? need : int64_t(sms) * 16);
  const size_t esm = sizeof(double) * sp.ndim * (sp.nbins + 1);
  const size_t sm = UuxHelLayout::total(2 + sp.ndim * sp.nbins);
  if (precision == 0) {
    RecordView<double> rec = RecordView<double>::carve(rec_base, sp.n_final, sp.ndim, C);
    e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    k_sample_rec<double><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);
    if (ev) cudaEventRecord(ev[1], s);
    k_me_acc_uux_hel<double><<<grid, kThreads, sm, s>>>(mp, sp.ndim, sp.nbins, rec, accumulate, partials, counters,
                                                        w_out, seed, iter, first_event, hel_T, hel_sq);
  } else {
    RecordView<float> rec = RecordView<float>::carve(rec_base, sp.n_final, sp.ndim, C);
    e = cudaMemsetAsync(rec.count, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[0], s);
    k_sample_rec<float><<<sgrid, kThreads, esm, s>>>(sp, edges, first_event, n, seed, iter, rec, w_out);
    if (ev) cudaEventRecord(ev[1], s);
    k_me_acc_uux_hel<float><<<grid, kThreads, sm, s>>>(mp, sp.ndim, sp.nbins, rec, accumulate, partials, counters,
                                                       w_out, seed, iter, first_event, hel_T, hel_sq);
  }
  if (ev) cudaEventRecord(ev[2], s);
  return cudaGetLastError();
}

}  // namespace mf
