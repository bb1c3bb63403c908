// Host side of the split-step path: FP64 construction of the per-step spectral
// tables of the channel and of DBP (stored as head/tail float pairs), the
// unit-modulus twiddle tables of the cluster transform, a per-device cache of
// both, and the C ABI entry points ssm_forward / dbp_apply.
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "ssm.cuh"
#include "ssm_host.cuh"

namespace ldbp {

static const double kPi = 3.14159265358979323846;
static const double kPlanck = 6.626e-34;  // Table I

FiberSI to_si(const ldbp_fiber& f) {
  FiberSI s;
  s.alpha = f.alpha_db_per_km * std::log(10.0) / 10.0 / 1e3;
  s.beta2 = f.beta2_ps2_per_km * 1e-27;
  s.gamma = f.gamma_per_w_km * 1e-3;
  return s;
}

double leff(double alpha, double z) { return alpha == 0.0 ? z : -std::expm1(-alpha * z) / alpha; }
double lmid(double alpha, double z) { return alpha == 0.0 ? z : 2.0 * std::sinh(alpha * z / 2.0) / alpha; }

// exp(j (beta2/2) w_k^2 z) e^{-alpha z / 2} / n on the fftfreq grid (Eq. (5)).
static std::vector<std::complex<double>> dispersion_table(long long n, double fs, double beta2, double alpha,
                                                          double z) {
  std::vector<std::complex<double>> t((size_t)n);
  const double amp = std::exp(-alpha * z / 2.0) / (double)n;
  for (long long k = 0; k < n; ++k) {
    const double kk = (double)(k < (n + 1) / 2 ? k : k - n);
    const double w = 2.0 * kPi * fs * kk / (double)n;
    const double ph = beta2 / 2.0 * w * w * z;
    t[(size_t)k] = std::polar(amp, ph);
  }
  return t;
}

SsmProgram build_channel(const ldbp_fiber& f, const ldbp_link& l, double fs, long long n) {
  const FiberSI s = to_si(f);
  const double Lsp = l.span_km * 1e3;
  const int N = l.steps_per_span;
  const double d = Lsp / N;
  const double G = std::exp(s.alpha * Lsp / 2.0);
  SsmProgram p;
  if (l.ase) {
    const double nf = std::pow(10.0, l.nf_db / 10.0);
    const double g = std::exp(s.alpha * Lsp);
    const double nsp = nf / (2.0 * (1.0 - 1.0 / g));
    const double psd = (g - 1.0) * kPlanck * l.carrier_hz * nsp;
    p.noise_std = std::sqrt((double)n * psd * fs / 2.0);
  }
  const int16_t no_noise = -2;
  if (l.symmetric) {
    p.tabs.push_back(dispersion_table(n, fs, s.beta2, s.alpha, d / 2.0));  // 0: half step
    p.tabs.push_back(dispersion_table(n, fs, s.beta2, s.alpha, d));        // 1: full step
    const float c = (float)(s.gamma * lmid(s.alpha, d));
    p.steps.push_back({0, no_noise, 0, 1.0f, c});
    for (int sp = 0; sp < l.n_spans; ++sp)
      for (int i = 0; i < N; ++i) {
        if (sp == 0 && i == 0) continue;
        if (i == 0)  // span boundary: half step, amplifier (+ ASE), half step
          p.steps.push_back({1, (int16_t)(l.ase ? 0 : no_noise), sp - 1, (float)G, c});
        else
          p.steps.push_back({1, no_noise, 0, 1.0f, c});
      }
    p.steps.push_back({0, (int16_t)(l.ase ? -1 : no_noise), l.n_spans - 1, (float)G, 0.0f});
  } else {
    p.tabs.push_back(dispersion_table(n, fs, s.beta2, s.alpha, d));  // 0: full step
    const float c = (float)(s.gamma * leff(s.alpha, d));
    p.c_pre = c;
    const int total = l.n_spans * N;
    for (int g = 0; g < total; ++g) {
      const bool end = (g + 1) % N == 0;
      p.steps.push_back({0, (int16_t)(end && l.ase ? -1 : no_noise), g / N, end ? (float)G : 1.0f,
                         g == total - 1 ? 0.0f : c});
    }
  }
  return p;
}

SsmProgram build_dbp(const ldbp_fiber& f, const ldbp_link& l, double fs, long long n, int N, bool symmetric) {
  const FiberSI s = to_si(f);
  const double Lsp = l.span_km * 1e3;
  const double d = Lsp / N;
  const double Ginv = std::exp(-s.alpha * Lsp / 2.0);
  SsmProgram p;
  const int16_t no_noise = -2;
  if (symmetric) {
    p.tabs.push_back(dispersion_table(n, fs, -s.beta2, -s.alpha, d / 2.0));
    p.tabs.push_back(dispersion_table(n, fs, -s.beta2, -s.alpha, d));
    const float c = (float)(-s.gamma * lmid(s.alpha, d));
    p.steps.push_back({0, no_noise, 0, (float)Ginv, c});
    for (int sp = 0; sp < l.n_spans; ++sp)
      for (int i = 0; i < N; ++i) {
        if (sp == 0 && i == 0) continue;
        p.steps.push_back({1, no_noise, 0, i == 0 ? (float)Ginv : 1.0f, c});
      }
    p.steps.push_back({0, no_noise, 0, 1.0f, 0.0f});
  } else {
    p.tabs.push_back(dispersion_table(n, fs, -s.beta2, -s.alpha, d));
    const float c = (float)(-s.gamma * leff(s.alpha, d));
    const int total = l.n_spans * N;
    for (int g = 0; g < total; ++g) p.steps.push_back({0, no_noise, 0, g % N == 0 ? (float)Ginv : 1.0f, c});
  }
  return p;
}

// ---------------------------------------------------------------- device cache
static std::mutex g_cache_mu;
static std::map<std::string, std::shared_ptr<DeviceProgram>> g_programs;
static std::map<std::string, float2*> g_twiddles;

template <typename T>
static cudaError_t upload(const std::vector<T>& h, T** out) {
  cudaError_t e = cudaMalloc(out, h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Spectral table as a float head per value (the float rounding of each part)
// and a tail: the remainder value - head divided by `scale` (the largest
// remainder of the table) as a half2.  Head plus tail carry about 36 bits;
// the split-step kernel multiplies by the same table at every step, so the
// head's rounding alone would add up coherently over a long run.
static cudaError_t upload_table(const std::vector<std::complex<double>>& v, float2** head, uint32_t** tail,
                                float* scale) {
  std::vector<float2> h(v.size());
  std::vector<double> lo(2 * v.size());
  double m = 0.0;
  for (size_t i = 0; i < v.size(); ++i) {
    const double re = v[i].real(), im = v[i].imag();
    h[i] = make_float2((float)re, (float)im);
    lo[2 * i] = re - (double)h[i].x;
    lo[2 * i + 1] = im - (double)h[i].y;
    m = std::max(m, std::max(std::fabs(lo[2 * i]), std::fabs(lo[2 * i + 1])));
  }
  *scale = m > 0.0 ? (float)m : 1.0f;
  std::vector<uint32_t> t(v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    const __half2 q = __floats2half2_rn((float)(lo[2 * i] / *scale), (float)(lo[2 * i + 1] / *scale));
    memcpy(&t[i], &q, sizeof(uint32_t));
  }
  cudaError_t e = upload(h, head);
  if (e != cudaSuccess) return e;
  return upload(t, tail);
}

// A float pair (c, s) close to (cos t, sin t) = w with c^2 + s^2 as close to 1
// as the float grid allows near w.  Candidates: one part moved by up to
// kUnitSteps float steps from its rounding, the other the float rounding of
// sqrt(1 - part^2) or a neighbour of it; the pair with the smallest
// |c^2 + s^2 - 1| (evaluated exactly in double) within kUnitMaxDist of w wins,
// the plain rounding when nothing beats it.  A twiddle of modulus 1 applied
// forward and its conjugate applied in the inverse transform cancel exactly,
// so its angle error does not build up over the steps of a long run.
static float2 unit_float2(double c, double s) {
  constexpr int kUnitSteps = 8;
  constexpr double kUnitMaxDist = 2e-6;
  float2 best = make_float2((float)c, (float)s);
  auto res = [](float x, float y) { return std::fabs((double)x * x + (double)y * y - 1.0); };
  double bres = res(best.x, best.y);
  for (int role = 0; role < 2; ++role) {
    const double a_true = role == 0 ? c : s, o_true = role == 0 ? s : c;
    float a = (float)a_true;
    for (int k = 0; k < kUnitSteps; ++k) a = std::nextafter(a, -2.0f);
    for (int k = -kUnitSteps; k <= kUnitSteps; ++k, a = std::nextafter(a, 2.0f)) {
      const double rem = 1.0 - (double)a * (double)a;
      if (rem < 0.0) continue;
      const float o0 = (float)std::copysign(std::sqrt(rem), o_true);
      const float cand[3] = {std::nextafter(o0, -2.0f), o0, std::nextafter(o0, 2.0f)};
      for (float o : cand) {
        const float x = role == 0 ? a : o, y = role == 0 ? o : a;
        const double dist = std::hypot((double)x - c, (double)y - s);
        const double r = res(x, y);
        if (dist <= kUnitMaxDist && r < bres) {
          best = make_float2(x, y);
          bres = r;
        }
      }
    }
  }
  return best;
}

int get_twiddle(long long n, int P, int log_n2, float2** out) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  const std::string key = std::to_string(dev) + ":" + std::to_string(n) + ":" + std::to_string(P);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_twiddles.find(key);
  if (it != g_twiddles.end()) {
    *out = it->second;
    return 0;
  }
  const long long N2 = 1LL << log_n2;
  std::vector<std::complex<double>> w((size_t)ssm_twiddle_count(P, log_n2));
  for (int q = 1; q < P; ++q)
    for (long long k2 = 0; k2 < N2; ++k2)
      w[(size_t)((q - 1) * N2 + k2)] = std::polar(1.0, -2.0 * kPi * (double)(q * k2) / (double)n);
  size_t off = (size_t)(P - 1) * (size_t)N2;
  for (int logns = 0; logns < log_n2;) {
    const int logr = (logns == 0 && (log_n2 % 4) != 0) ? (log_n2 % 4) : 4;
    const long long Ns = 1LL << logns, R = 1LL << logr;
    if (logns > 0) {
      for (long long q = 1; q < R; ++q)
        for (long long k = 0; k < Ns; ++k)
          w[off + (size_t)((q - 1) * Ns + k)] = std::polar(1.0, -2.0 * kPi * (double)(q * k) / (double)(Ns * R));
      off += (size_t)((R - 1) * Ns);
    }
    logns += logr;
  }
  std::vector<float2> wf(w.size());
  for (size_t i = 0; i < w.size(); ++i) wf[i] = unit_float2(w[i].real(), w[i].imag());
  float2* d = nullptr;
  cudaError_t e = upload(wf, &d);
  if (e != cudaSuccess) return cuda_fail(e, "twiddle table");
  g_twiddles[key] = d;
  *out = d;
  return 0;
}

int get_program(const std::string& key_in, const SsmProgram& prog, std::shared_ptr<DeviceProgram>* out) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  const std::string key = std::to_string(dev) + "|" + key_in;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_programs.find(key);
  if (it != g_programs.end()) {
    *out = it->second;
    return 0;
  }
  auto dp = std::make_shared<DeviceProgram>();
  for (const auto& t : prog.tabs) {
    float2* d = nullptr;
    uint32_t* dl = nullptr;
    float sc = 1.f;
    cudaError_t e = upload_table(t, &d, &dl, &sc);
    if (e != cudaSuccess) return cuda_fail(e, "ssm table");
    dp->tabs.push_back(d);
    dp->tabs_lo.push_back(dl);
    dp->tabs_lo_scale.push_back(sc);
  }
  cudaError_t e = cudaMalloc(&dp->steps, prog.steps.size() * sizeof(SsmStep));
  if (e != cudaSuccess) return cuda_fail(e, "ssm steps");
  e = cudaMemcpy(dp->steps, prog.steps.data(), prog.steps.size() * sizeof(SsmStep), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "ssm steps copy");
  dp->nsteps = (int)prog.steps.size();
  dp->host_steps = prog.steps;
  dp->c_pre = (float)prog.c_pre;
  dp->noise_std = (float)prog.noise_std;
  g_programs[key] = dp;
  *out = dp;
  return 0;
}

static std::string fkey(const ldbp_fiber& f, double fs, long long n) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%.17g,%.17g,%.17g,%.17g,%lld", f.alpha_db_per_km, f.beta2_ps2_per_km,
           f.gamma_per_w_km, fs, n);
  return buf;
}

int check_link(const ldbp_fiber* f, const ldbp_link* l, double fs, const void* x, const void* y, long long n,
               int batch, bool pow2) {
  if (!f || !l || !x || !y) return fail(LDBP_EINVAL, "fiber, link, x and y must be non-NULL");
  if (!std::isfinite(fs)) return fail(LDBP_ENONFINITE, "fs_hz is NaN or infinite");
  if (!(fs > 0.0)) return fail(LDBP_EINVAL, "fs_hz must be positive");
  if (!std::isfinite(f->alpha_db_per_km) || !std::isfinite(f->beta2_ps2_per_km) || !std::isfinite(f->gamma_per_w_km) ||
      !std::isfinite(l->span_km) || !std::isfinite(l->nf_db) || !std::isfinite(l->carrier_hz))
    return fail(LDBP_ENONFINITE, "fiber or link parameter is NaN or infinite");
  if (f->alpha_db_per_km < 0) return fail(LDBP_EINVAL, "alpha must be >= 0");
  if (l->n_spans < 1 || !(l->span_km > 0.0) || l->steps_per_span < 1)
    return fail(LDBP_EINVAL, "link needs n_spans >= 1, span_km > 0, steps_per_span >= 1");
  if (batch < 1) return fail(LDBP_EINVAL, "batch=%d must be >= 1", batch);
  if (!pow2) {
    if (n < 2 || n > (1LL << 27)) return fail(LDBP_EINVAL, "n=%lld must be in [2, 2^27]", n);
  } else {
    const bool three = n % 3 == 0;
    const long long m = three ? n / 3 : n;
    const long long lo = three ? (1LL << 9) : (1LL << kSsmMinLogN2), hi = three ? (1LL << 14) : (1LL << (kSsmMaxLogN2 + 4));
    if (m < lo || m > hi || (m & (m - 1)))
      return fail(LDBP_EINVAL, "n=%lld must be a power of two in [%d, %d] or three times one in [%d, %d]", n,
                  1 << kSsmMinLogN2, 1 << (kSsmMaxLogN2 + 4), 3 << 9, 3 << 14);
  }
  if ((long long)l->n_spans * l->steps_per_span > 1000000) return fail(LDBP_EINVAL, "too many steps");
  return 0;
}

int run_program(const DeviceProgram& dp, const void* x, void* y, long long n, int batch, const float* wave_scale,
                int wave_mode, uint64_t seed, uint64_t counter, cudaStream_t st) {
  // Larger batches of n = 65536 and 131072 run on the L2-resident two-kernel
  // path: a waveform would need a 16-block cluster, and few such clusters fit
  // on the GPU at once.
  if (!wave_scale && ssm_stream_preferred(n, batch))
    return run_program_stream(dp, x, y, n, batch, seed, counter, st);
  int sms = 0, dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  LDBP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int P = 1, log_n2 = 0;
  if (ssm_choose_cluster(n, batch, sms, &P, &log_n2)) return fail(LDBP_EINVAL, "unsupported n=%lld", n);
  float2* tw = nullptr;
  if (int rc = get_twiddle(n, P, log_n2, &tw)) return rc;
  SsmParams p;
  memset(&p, 0, sizeof(p));
  p.x = static_cast<const float2*>(x);
  p.y = static_cast<float2*>(y);
  p.n = n;
  p.batch = batch;
  p.nsteps = dp.nsteps;
  p.steps = dp.steps;
  for (size_t i = 0; i < dp.tabs.size() && i < (size_t)kSsmMaxTabs; ++i) {
    p.tabs[i] = dp.tabs[i];
    p.tabs_lo[i] = dp.tabs_lo[i];
    p.tabs_lo_scale[i] = dp.tabs_lo_scale[i];
  }
  p.twiddle = tw;
  p.wave_scale = wave_scale;
  p.wave_mode = wave_mode;
  p.c_pre = dp.c_pre;
  p.noise_std = dp.noise_std;
  p.seed_lo = (uint32_t)(seed & 0xffffffffu);
  p.seed_hi = (uint32_t)(seed >> 32);
  p.counter = (uint32_t)(counter & 0xffffffffu);
  cudaError_t e = launch_ssm(p, P, log_n2, st);
  if (e != cudaSuccess) return cuda_fail(e, "ssm launch");
  return 0;
}

int link_program(const ldbp_fiber& f, const ldbp_link& l, double fs, long long n, int dbp_steps, bool dbp_symmetric,
                 std::shared_ptr<DeviceProgram>* out) {
  char buf[256];
  if (dbp_steps == 0)
    snprintf(buf, sizeof(buf), "ch|%d,%.17g,%d,%d,%d,%.17g,%.17g", l.n_spans, l.span_km, l.steps_per_span,
             l.symmetric ? 1 : 0, l.ase ? 1 : 0, l.nf_db, l.carrier_hz);
  else
    snprintf(buf, sizeof(buf), "dbp|%d,%.17g,%d,%d", l.n_spans, l.span_km, dbp_steps, dbp_symmetric ? 1 : 0);
  const std::string key = fkey(f, fs, n) + buf;
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  bool need = true;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    need = g_programs.find(std::to_string(dev) + "|" + key) == g_programs.end();
  }
  SsmProgram prog;
  if (need) prog = dbp_steps == 0 ? build_channel(f, l, fs, n) : build_dbp(f, l, fs, n, dbp_steps, dbp_symmetric);
  return get_program(key, prog, out);
}

}  // namespace ldbp

using namespace ldbp;

extern "C" {

int ssm_forward(const ldbp_fiber* fiber, const ldbp_link* link, double fs_hz, const void* x, void* y, int64_t n,
                int32_t batch, void* stream) {
  if (int rc = check_link(fiber, link, fs_hz, x, y, n, batch)) return rc;
  std::shared_ptr<DeviceProgram> dp;
  if (int rc = link_program(*fiber, *link, fs_hz, n, 0, false, &dp)) return rc;
  return run_program(*dp, x, y, n, batch, nullptr, 0, link->seed, link->counter, static_cast<cudaStream_t>(stream));
}

int dbp_apply(const ldbp_fiber* fiber, const ldbp_link* link, double fs_hz, int32_t steps_per_span,
              int32_t symmetric, const void* x, void* y, int64_t n, int32_t batch, void* stream) {
  if (int rc = check_link(fiber, link, fs_hz, x, y, n, batch)) return rc;
  if (steps_per_span < 1) return fail(LDBP_EINVAL, "steps_per_span=%d must be >= 1", steps_per_span);
  std::shared_ptr<DeviceProgram> dp;
  if (int rc = link_program(*fiber, *link, fs_hz, n, steps_per_span, symmetric != 0, &dp)) return rc;
  return run_program(*dp, x, y, n, batch, nullptr, 0, 0, 0, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
