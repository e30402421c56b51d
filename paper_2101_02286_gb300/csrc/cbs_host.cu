// cbs_host.cu -- solves from host memory: a pipe of plans over one field,
// copies in and out inside the call (cbs_pipe_* in cbs.h).
//
// Per call, with buffer set b = call % 2:
//   upload stream:  h_in -> d_in[b] (after the solves of call - 2 have read d_in[b]);
//   caller's stream: every plan's solve d_in[b] -> d_out[b][k];
//   download stream: d_out[b][k] -> h_out[k] as soon as solve k is done;
//   the caller's stream then waits for the downloads, so work issued on it
//   after the call (or a synchronize) sees the results on the host.
// The upload of call i + 1 runs on its own copy engine while call i's
// results travel back.
#include <cuda_runtime.h>

#include <new>
#include <string>
#include <vector>

#include "cbs_plan_struct.h"

struct cbs_pipe {
  std::vector<cbs_plan*> plans;
  size_t in_bytes = 0;
  std::vector<size_t> out_bytes;
  void* d_in[2] = {nullptr, nullptr};
  std::vector<void*> d_out[2];
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t up_done[2] = {nullptr, nullptr}, comp_done[2] = {nullptr, nullptr}, down_done[2] = {nullptr, nullptr};
  std::vector<cudaEvent_t> solved[2];
  bool used[2] = {false, false};
  int device = -1;
  long long calls = 0;
};

namespace {

size_t elem_size(int dtype) { return dtype == CBS_DTYPE_F64 ? 8 : 4; }

void release(cbs_pipe* S) {
  for (int b = 0; b < 2; b++) {
    if (S->d_in[b]) cudaFree(S->d_in[b]);
    for (void* p : S->d_out[b])
      if (p) cudaFree(p);
    for (cudaEvent_t e : S->solved[b])
      if (e) cudaEventDestroy(e);
    if (S->up_done[b]) cudaEventDestroy(S->up_done[b]);
    if (S->comp_done[b]) cudaEventDestroy(S->comp_done[b]);
    if (S->down_done[b]) cudaEventDestroy(S->down_done[b]);
  }
  if (S->up) cudaStreamDestroy(S->up);
  if (S->down) cudaStreamDestroy(S->down);
  delete S;
}

}  // namespace

extern "C" {

cbs_status cbs_pipe_create(cbs_pipe** out, cbs_plan* const* plans, int32_t count) {
  using namespace cbs;
  if (!out || !plans || count < 1 || count > 64) return set_error(CBS_ERR_INVALID_ARG, "pipe: 1..64 plans");
  *out = nullptr;
  const cbs_desc& d0 = plans[0] ? plans[0]->desc : cbs_desc{};
  for (int k = 0; k < count; k++) {
    if (!plans[k]) return set_error(CBS_ERR_INVALID_ARG, "pipe: null plan");
    const cbs_desc& d = plans[k]->desc;
    if (d.dims[0] != d0.dims[0] || d.dims[1] != d0.dims[1] || d.dims[2] != d0.dims[2] || d.in_dtype != d0.in_dtype)
      return set_error(CBS_ERR_INVALID_ARG, "pipe: every plan reads the same field (dims and input type)");
  }
  cbs_pipe* S = new (std::nothrow) cbs_pipe();
  if (!S) return set_error(CBS_ERR_NO_MEMORY, "host allocation failed");
  const size_t elems = (size_t)d0.dims[0] * d0.dims[1] * d0.dims[2];
  S->in_bytes = elems * elem_size(d0.in_dtype);
  for (int k = 0; k < count; k++) {
    S->plans.push_back(plans[k]);
    S->out_bytes.push_back(elems * elem_size(plans[k]->desc.out_dtype));
  }
  cudaError_t e = cudaGetDevice(&S->device);
  for (int b = 0; b < 2 && e == cudaSuccess; b++) {
    e = cudaMalloc(&S->d_in[b], S->in_bytes);
    S->d_out[b].assign(count, nullptr);
    S->solved[b].assign(count, nullptr);
    for (int k = 0; k < count && e == cudaSuccess; k++) e = cudaMalloc(&S->d_out[b][k], S->out_bytes[k]);
    for (int k = 0; k < count && e == cudaSuccess; k++)
      e = cudaEventCreateWithFlags(&S->solved[b][k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->up_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->comp_done[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->down_done[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->up, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->down, cudaStreamNonBlocking);
  // touch every buffer once, so that the first calls do not pay for backing
  // fresh device memory inside their copies
  for (int b = 0; b < 2 && e == cudaSuccess; b++) {
    e = cudaMemsetAsync(S->d_in[b], 0, S->in_bytes, S->up);
    for (int k = 0; k < count && e == cudaSuccess; k++) e = cudaMemsetAsync(S->d_out[b][k], 0, S->out_bytes[k], S->up);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(S->up);
  if (e != cudaSuccess) {
    release(S);
    return set_error(e == cudaErrorMemoryAllocation ? CBS_ERR_NO_MEMORY : CBS_ERR_CUDA,
                     std::string("pipe setup: ") + cudaGetErrorString(e));
  }
  *out = S;
  return CBS_OK;
}

cbs_status cbs_pipe_solve(cbs_pipe* S, const void* host_in, void* const* host_outs, void* stream) {
  using namespace cbs;
  set_launch_count(0);
  if (!S || !host_in || !host_outs) return set_error(CBS_ERR_INVALID_ARG, "null argument");
  for (size_t k = 0; k < S->plans.size(); k++)
    if (!host_outs[k]) return set_error(CBS_ERR_INVALID_ARG, "pipe: null output " + std::to_string(k));
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != S->device)
    return set_error(CBS_ERR_INVALID_ARG, "pipe: call it with the device it was created on current");
  const cudaStream_t s = (cudaStream_t)stream;
  const int b = (int)(S->calls & 1);
  auto cuda = [&](cudaError_t e, const char* what) -> cbs_status {
    return e == cudaSuccess ? CBS_OK : set_error(CBS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cbs_status st;
  // upload, once the solves of the call before last have read d_in[b]
  if (S->used[b] && (st = cuda(cudaStreamWaitEvent(S->up, S->comp_done[b], 0), "pipe wait"))) return st;
  if ((st = cuda(cudaMemcpyAsync(S->d_in[b], host_in, S->in_bytes, cudaMemcpyHostToDevice, S->up), "pipe upload")))
    return st;
  if ((st = cuda(cudaEventRecord(S->up_done[b], S->up), "pipe event"))) return st;
  // solves on the caller's stream, once the input is there and d_out[b] is free
  if ((st = cuda(cudaStreamWaitEvent(s, S->up_done[b], 0), "pipe wait"))) return st;
  if (S->used[b] && (st = cuda(cudaStreamWaitEvent(s, S->down_done[b], 0), "pipe wait"))) return st;
  int launches = 0;
  for (size_t k = 0; k < S->plans.size(); k++) {
    st = cbs_solve(S->plans[k], S->d_in[b], S->d_out[b][k], stream);
    if (st) return st;
    launches += cbs_last_launch_count();
    if ((st = cuda(cudaEventRecord(S->solved[b][k], s), "pipe event"))) return st;
  }
  if ((st = cuda(cudaEventRecord(S->comp_done[b], s), "pipe event"))) return st;
  // downloads, each as soon as its solve is done
  for (size_t k = 0; k < S->plans.size(); k++) {
    if ((st = cuda(cudaStreamWaitEvent(S->down, S->solved[b][k], 0), "pipe wait"))) return st;
    if ((st = cuda(cudaMemcpyAsync(host_outs[k], S->d_out[b][k], S->out_bytes[k], cudaMemcpyDeviceToHost, S->down),
                   "pipe download")))
      return st;
  }
  if ((st = cuda(cudaEventRecord(S->down_done[b], S->down), "pipe event"))) return st;
  if ((st = cuda(cudaStreamWaitEvent(s, S->down_done[b], 0), "pipe wait"))) return st;
  S->used[b] = true;
  S->calls++;
  set_launch_count(launches);
  return CBS_OK;
}

cbs_status cbs_pipe_destroy(cbs_pipe* S) {
  if (!S) return cbs::set_error(CBS_ERR_INVALID_ARG, "null pipe");
  cudaDeviceSynchronize();
  release(S);
  return CBS_OK;
}

}  // extern "C"
