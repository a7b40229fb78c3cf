// owqs_run_static: the simulation entry point for callers that cannot
// allocate device memory.  Its scratch (ping-pong state buffers, norm slots,
// reduction partials and the finished-block counter) lives in one file-scope
// device array instead of cudaMalloc'd memory.  The caller passes the input
// and output vectors as with owqs_run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "owqs_internal.h"

namespace owqs {

// header: counter, block partials, norm slots; then two equal state buffers
constexpr size_t kStaticHeaderBytes = 256u << 10;
constexpr size_t kStaticBufferBytes = 4u << 20;
constexpr size_t kStaticScratchBytes = kStaticHeaderBytes + 2 * kStaticBufferBytes;
constexpr size_t kStaticPartialsOffset = 256;
constexpr size_t kStaticPartialsBytes = 2u * 8u * 1024u * sizeof(double);  // up to 1024 SMs
constexpr size_t kStaticNormsOffset = kStaticPartialsOffset + kStaticPartialsBytes;

static __device__ __align__(256) unsigned char g_owqs_static_scratch[kStaticScratchBytes];

// Device address of the scratch array, looked up once per device with that
// device current.  In host code the array's name is only a host-side stand-in.
static owqs_status static_scratch(unsigned char** out) {
  static std::mutex mu;
  static std::vector<unsigned char*> addr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(OWQS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(mu);
  if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_owqs_static_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return set_error(OWQS_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") +
                                          cudaGetErrorString(e));
    }
    addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = addr[dev];
  return OWQS_OK;
}

namespace {

struct StaticSource : OutcomeSource {
  const Pattern& p;
  const uint8_t* bits;  // nullptr => all zero
  StaticSource(const Pattern& pp, const uint8_t* b) : p(pp), bits(b) {}
  bool known_upfront(std::vector<int8_t>& o) override {
    for (size_t k = 0; k < p.meas_qubit.size(); ++k) o[p.meas_qubit[k]] = bits ? (int8_t)(bits[k] & 1u) : 0;
    return true;
  }
  int decide(const PassDesc& d) override { return bits ? (bits[d.meas_k] & 1u) : 0; }
};

owqs_status cuda_err(cudaError_t e, const char* what) {
  cudaGetLastError();
  return set_error(OWQS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

static owqs_status run_static(Pattern& p, const owqs_run_opts* o, const void* psi_in, void* psi_out,
                              uint8_t* outcomes, double* probs) {
  if (!o || !psi_out) return set_error(OWQS_ERR_ARG, "NULL argument");
  if (o->dtype > OWQS_C128 || o->mode > OWQS_MODE_EOWQS) return set_error(OWQS_ERR_ARG, "bad option value");
  if (o->io != OWQS_IO_DEVICE) return set_error(OWQS_ERR_ARG, "owqs_run_static takes device vectors only");
  if (o->policy != OWQS_OUTCOME_FORCED && o->policy != OWQS_OUTCOME_ZERO)
    return set_error(OWQS_ERR_UNSUPPORTED, "owqs_run_static takes forced or zero outcomes");
  if (o->policy == OWQS_OUTCOME_FORCED && !outcomes && !p.meas_qubit.empty())
    return set_error(OWQS_ERR_ARG, "forced outcomes need the outcomes array");
  if (((uintptr_t)psi_in % 16) || ((uintptr_t)psi_out % 16))
    return set_error(OWQS_ERR_ARG, "device vectors must be 16-byte aligned");
  const int dtype = (int)o->dtype, mode = (int)o->mode;
  const size_t amp = dtype == OWQS_C64 ? 8 : 16;
  if (psi_in && byte_ranges_overlap(psi_in, amp << p.inputs.size(), psi_out, amp << p.outputs.size()))
    return set_error(OWQS_ERR_ARG, "psi_in and psi_out must not overlap");
  const int K = (int)p.meas_qubit.size();

  StaticSource src(p, o->policy == OWQS_OUTCOME_ZERO ? nullptr : outcomes);
  std::vector<PassDesc> passes;
  owqs_status st = compile_schedule(p, mode, src, passes);
  if (st != OWQS_OK) return st;
  size_t widest = 1;
  for (const PassDesc& d : passes)
    if (d.kind == 0) widest = std::max<size_t>(widest, (size_t)1 << d.n_out);
  const size_t max_elems = kStaticBufferBytes / amp;
  if (widest > max_elems)
    return set_error(OWQS_ERR_ARG, "owqs_run_static: the widest pass needs " + std::to_string(widest) +
                                       " amplitudes per buffer; the static scratch holds " +
                                       std::to_string(max_elems) + " (" + std::to_string(kStaticBufferBytes) +
                                       " bytes per buffer)");
  const size_t nslots = 3 * (size_t)K + 8;
  if (kStaticNormsOffset + nslots * sizeof(double) > kStaticHeaderBytes)
    return set_error(OWQS_ERR_ARG, "owqs_run_static: too many measurements for the static norm slots");
  if ((size_t)max_grid() * 2 * sizeof(double) > kStaticPartialsBytes)
    return set_error(OWQS_ERR_UNSUPPORTED, "owqs_run_static: device has more SMs than the scratch provides for");

  unsigned char* base = nullptr;
  st = static_scratch(&base);
  if (st != OWQS_OK) return st;
  unsigned int* counter = reinterpret_cast<unsigned int*>(base);
  double* partials = reinterpret_cast<double*>(base + kStaticPartialsOffset);
  double* norms = reinterpret_cast<double*>(base + kStaticNormsOffset);
  void* buf[2] = {base + kStaticHeaderBytes, base + kStaticHeaderBytes + kStaticBufferBytes};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(o->stream);
  const double thresh = dtype == OWQS_C128 ? 1e-24 : 1e-12;

  // the array keeps the previous call's contents: the counter and the error
  // flag after it must start at 0
  cudaError_t e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_err(e, "clearing the static counter");

  const uint64_t in_elems = 1ull << p.inputs.size();
  const void* cur = psi_in;
  int prev = -1;
  if (psi_in) {
    const int grid = (int)std::min<uint64_t>((in_elems + kBlock - 1) / kBlock, (uint64_t)max_grid());
    e = launch_norm(psi_in, in_elems, dtype, norms, 0, partials, counter, grid, s);
    if (e != cudaSuccess) return cuda_err(e, "norm kernel");
    if (mode == OWQS_MODE_OWQS) prev = 0;
  }
  int i = 0;
  for (const PassDesc& d : passes) {
    PassParams P;
    LaunchPlan L;
    plan_pass(d, dtype, cur == nullptr, P, L);
    P.norms = norms;
    P.partials = partials;
    P.counter = counter;
    P.errflag = counter + 1;
    P.thresh = thresh;
    P.in = cur;
    P.in_cap = cur == nullptr ? 0 : (cur == psi_in ? in_elems : max_elems);
    if (d.kind == 0) {
      P.out = buf[i & 1];
      P.out_cap = max_elems;
      P.norm_in = prev;
      P.norm_out = mode == OWQS_MODE_OWQS ? i + 1 : -1;
      prev = P.norm_out;
      ++i;
    } else {
      P.out = psi_out;
      P.out_cap = 1ull << p.outputs.size();
      P.norm_in = mode == OWQS_MODE_OWQS ? prev : -1;
      P.norm_out = K + 1;
    }
    e = launch_pass(P, L, dtype, s);
    if (e != cudaSuccess) return cuda_err(e, "pass kernel");
    cur = P.out;
  }
  std::vector<double> h((size_t)K + 2, 0.0);
  unsigned int flag = 0;
  e = cudaMemcpyAsync(h.data(), norms, sizeof(double) * (K + 2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, counter + 1, sizeof(flag), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "static run");
  if (flag & 2u)
    return set_error(OWQS_ERR_CUDA, "a kernel access fell outside its buffer (bounds-checked build); results are invalid");
  if (flag) return set_error(OWQS_ERR_TIMEOUT, "a device-side wait in a pass kernel gave up; results are invalid");

  st = OWQS_OK;
  int mi = 0;
  for (const PassDesc& d : passes) {
    if (d.kind != 0) continue;
    const double pv = mode == OWQS_MODE_OWQS ? h[mi + 1] : 0.5;
    if (probs) probs[d.meas_k] = pv;
    if (outcomes && o->policy == OWQS_OUTCOME_ZERO) outcomes[d.meas_k] = 0;
    if (mode == OWQS_MODE_OWQS && !(pv >= thresh) && st == OWQS_OK)
      st = set_error(OWQS_ERR_IMPOSSIBLE_BRANCH, "outcome of measurement " + std::to_string(d.meas_k) +
                                                      " has probability " + std::to_string(pv));
    ++mi;
  }
  if (mode == OWQS_MODE_EOWQS) {
    const double nin = psi_in ? h[0] : 1.0, nout = h[K + 1];
    const double tol = dtype == OWQS_C128 ? 1e-10 : 1e-4;
    if (!(std::fabs(nout - nin) <= tol * std::max(nin, 1e-300)))
      st = set_error(OWQS_ERR_NOT_DETERMINISTIC, "EOWQS output norm " + std::to_string(nout) +
                                                     " differs from the input norm " + std::to_string(nin));
  }
  return st;
}

}  // namespace owqs

extern "C" owqs_status owqs_run_static(owqs_pattern* h, const owqs_run_opts* opts, const void* psi_in,
                                       void* psi_out, uint8_t* outcomes, double* probs) {
  owqs::clear_error();
  if (!h) return owqs::set_error(OWQS_ERR_ARG, "NULL pattern");
  return owqs::run_static(h->p, opts, psi_in, psi_out, outcomes, probs);
}
