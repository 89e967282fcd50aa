// host_query.cu -- queries for baskets in host memory: chunked streaming through
// device staging slots with copies in, evaluation and copies out overlapped.
//
// Three streams of the pipeline: `in` (host -> device), `comp` (the query pass) and
// `out` (device -> host).  Chunk c uses slot c mod S.  Its input copy waits until
// the slot's previous chunk was evaluated (the inputs are free), its evaluation
// waits for its input copy and for the slot's previous output copy (the outputs
// are free), its output copy waits for its evaluation.  Events carry every
// dependency; nothing synchronises the host.  A call waits for the caller's stream as it
// was when the call was made; the caller's stream waits for the pipeline only at
// gv_pipeline_join, so consecutive calls keep the copy engines busy across baskets.
#include <new>
#include "gv_internal.h"

struct gv_pipeline {
  static constexpr int kMaxSlots = 8;
  struct Slot {
    double* in[6];         // x y z dx dy dz
    int8_t* code;
    double* res[4];        // dist_in dist_out safety_in safety_out
    uint32_t* idx;         // refinement worklist
    unsigned long long* counter;
    cudaEvent_t in_ready, comp_done, out_done;
    bool used;
  };
  int device;
  int64_t chunk;
  int slots;
  int next;
  void* mem;
  cudaStream_t s_in, s_comp, s_out;
  cudaEvent_t start, fin;
  Slot slot[kMaxSlots];
};

namespace gv {
namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

void release(gv_pipeline* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  for (int k = 0; k < p->slots; k++) {
    gv_pipeline::Slot& S = p->slot[k];
    if (S.in_ready) cudaEventDestroy(S.in_ready);
    if (S.comp_done) cudaEventDestroy(S.comp_done);
    if (S.out_done) cudaEventDestroy(S.out_done);
  }
  if (p->start) cudaEventDestroy(p->start);
  if (p->fin) cudaEventDestroy(p->fin);
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_comp) cudaStreamDestroy(p->s_comp);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  if (p->mem) cudaFree(p->mem);
  cudaSetDevice(cur);
  delete p;
}

}  // namespace
}  // namespace gv

using namespace gv;

gv_status gv_pipeline_create(int64_t chunk_tracks, int32_t slots, gv_pipeline** out) {
  if (!out) return set_error(GV_ERR_INVALID_ARG, "NULL output handle");
  *out = nullptr;
  if (chunk_tracks < 1 || chunk_tracks > (int64_t(1) << 31))
    return set_error(GV_ERR_INVALID_ARG, "chunk_tracks must be in [1, 2^31]");
  if (slots < 2 || slots > gv_pipeline::kMaxSlots) return set_error(GV_ERR_INVALID_ARG, "slots must be in [2, 8]");
  gv_pipeline* p = new (std::nothrow) gv_pipeline();
  if (!p) return set_error(GV_ERR_OUT_OF_MEMORY, "host allocation failed");
  p->chunk = chunk_tracks;
  p->slots = slots;
  p->next = 0;
  cudaError_t e = cudaGetDevice(&p->device);
  const size_t m = (size_t)chunk_tracks;
  const size_t per_slot = 6 * align256(8 * m) + align256(m) + 4 * align256(8 * m) + align256(4 * m) + 256;
  if (e == cudaSuccess) e = cudaMalloc(&p->mem, per_slot * (size_t)slots);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fin, cudaEventDisableTiming);
  for (int k = 0; k < slots && e == cudaSuccess; k++) {
    gv_pipeline::Slot& S = p->slot[k];
    char* base = static_cast<char*>(p->mem) + per_slot * (size_t)k;
    for (int j = 0; j < 6; j++) { S.in[j] = reinterpret_cast<double*>(base); base += align256(8 * m); }
    S.code = reinterpret_cast<int8_t*>(base); base += align256(m);
    for (int j = 0; j < 4; j++) { S.res[j] = reinterpret_cast<double*>(base); base += align256(8 * m); }
    S.idx = reinterpret_cast<uint32_t*>(base); base += align256(4 * m);
    S.counter = reinterpret_cast<unsigned long long*>(base);
    e = cudaEventCreateWithFlags(&S.in_ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.comp_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.out_done, cudaEventDisableTiming);
    S.used = false;
  }
  if (e != cudaSuccess) {
    release(p);
    return e == cudaErrorMemoryAllocation ? set_error(GV_ERR_OUT_OF_MEMORY, "cudaMalloc of the pipeline slots failed")
                                          : cuda_error(e, "gv_pipeline_create");
  }
  *out = p;
  return GV_OK;
}

void gv_pipeline_destroy(gv_pipeline* p) {
  if (!p) return;
  cudaStreamSynchronize(p->s_in);
  cudaStreamSynchronize(p->s_comp);
  cudaStreamSynchronize(p->s_out);
  release(p);
}

gv_status gv_query_host(const gv_solid* s, const gv_tracks* t, gv_precision prec, const gv_results* res,
                        gv_pipeline* p, void* stream) {
  const gv::Range range("gv_query_host");
  if (!s || !t || !res || !p) return set_error(GV_ERR_INVALID_ARG, "NULL solid, tracks, results or pipeline");
  if (t->n < 0) return set_error(GV_ERR_INVALID_ARG, "negative track count");
  if (prec != GV_FP64 && prec != GV_FP32_REFINE) return set_error(GV_ERR_INVALID_ARG, "unknown precision");
  if (t->n == 0) return GV_OK;
  const bool dirs = res->dist_in || res->dist_out;
  if (!t->x || !t->y || !t->z) return set_error(GV_ERR_INVALID_ARG, "NULL point array");
  if (dirs && (!t->dx || !t->dy || !t->dz)) return set_error(GV_ERR_INVALID_ARG, "distances requested without directions");
  const void* ptrs[10] = {t->x, t->y, t->z, t->dx, t->dy, t->dz, res->dist_in, res->dist_out, res->safety_in,
                          res->safety_out};
  for (int i = 0; i < 10; i++)
    if (ptrs[i] && ((uintptr_t)ptrs[i] & 7u)) return set_error(GV_ERR_INVALID_ARG, "arrays must be 8-byte aligned");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->device || s->device != p->device)
    return set_error(GV_ERR_INVALID_ARG, "pipeline, solid and current device differ");

  const double* hin[6] = {t->x, t->y, t->z, t->dx, t->dy, t->dz};
  double* hres[4] = {res->dist_in, res->dist_out, res->safety_in, res->safety_out};
  const int nin = dirs ? 6 : 3;
  cudaStream_t user = (cudaStream_t)stream;
  cudaError_t e = cudaEventRecord(p->start, user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_in, p->start, 0);
  for (int64_t off = 0; off < t->n && e == cudaSuccess; off += p->chunk) {
    const int64_t m = (t->n - off < p->chunk) ? t->n - off : p->chunk;
    gv_pipeline::Slot& S = p->slot[p->next];
    p->next = (p->next + 1) % p->slots;
    // copy in, once the slot's previous inputs have been consumed
    if (S.used) e = cudaStreamWaitEvent(p->s_in, S.comp_done, 0);
    for (int j = 0; j < nin && e == cudaSuccess; j++)
      e = cudaMemcpyAsync(S.in[j], hin[j] + off, 8 * (size_t)m, cudaMemcpyHostToDevice, p->s_in);
    if (e == cudaSuccess) e = cudaEventRecord(S.in_ready, p->s_in);
    // evaluate, once the inputs are in and the slot's previous results are out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_comp, S.in_ready, 0);
    if (e == cudaSuccess && S.used) e = cudaStreamWaitEvent(p->s_comp, S.out_done, 0);
    if (e == cudaSuccess) {
      QueryArgs a{S.in[0], S.in[1], S.in[2], dirs ? S.in[3] : nullptr, dirs ? S.in[4] : nullptr,
                  dirs ? S.in[5] : nullptr, res->inside ? S.code : nullptr,
                  hres[0] ? S.res[0] : nullptr, hres[1] ? S.res[1] : nullptr, hres[2] ? S.res[2] : nullptr,
                  hres[3] ? S.res[3] : nullptr, m};
      e = prec == GV_FP64 ? launch_query_fp64(s, a, p->s_comp) : launch_query_fp32(s, a, S.idx, S.counter, p->s_comp);
    }
    if (e == cudaSuccess) e = cudaEventRecord(S.comp_done, p->s_comp);
    // copy out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->s_out, S.comp_done, 0);
    if (e == cudaSuccess && res->inside)
      e = cudaMemcpyAsync(res->inside + off, S.code, (size_t)m, cudaMemcpyDeviceToHost, p->s_out);
    for (int j = 0; j < 4 && e == cudaSuccess; j++)
      if (hres[j]) e = cudaMemcpyAsync(hres[j] + off, S.res[j], 8 * (size_t)m, cudaMemcpyDeviceToHost, p->s_out);
    if (e == cudaSuccess) e = cudaEventRecord(S.out_done, p->s_out);
    S.used = true;
  }
  if (e != cudaSuccess) return cuda_error(e, "gv_query_host");
  return GV_OK;
}

gv_status gv_pipeline_join(gv_pipeline* p, void* stream) {
  if (!p) return set_error(GV_ERR_INVALID_ARG, "NULL pipeline");
  // the out stream is in order: its last copy is the end of every call made so far
  cudaError_t e = cudaEventRecord(p->fin, p->s_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, p->fin, 0);
  if (e != cudaSuccess) return cuda_error(e, "gv_pipeline_join");
  return GV_OK;
}
