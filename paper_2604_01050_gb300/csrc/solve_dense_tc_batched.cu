// solve_dense_tc_batched.cu -- the chunks of several small dense problems in
// one cooperative launch on the tensor cores (the parallel, independent
// repetitions of Sec. II B widened to many instances).
//
// Each problem of the batch runs the persistent tcgen05 solver of
// dense_tc_persistent.cuh (one CTA per 128 x 128 output tile, x and y in
// TMEM, per-tile step counters instead of a grid barrier) on its own tiles:
// CTAs tile0 .. tile0 + Mt * Ct - 1 of the launch, row-tile major.  A CTA
// finds its problem in a descriptor table that the host copies into device
// memory before the launch; the problem's tensor maps are read from there
// (fenced into the tensormap proxy first), its step counters sit in one flag
// array of the batch at offset tile0, and its error flag, step range and
// tables are its own, so a problem that stops early (its wait gave up, or
// its range ends) leaves the others running.  CTAs of one problem wait only
// on each other; the cooperative launch makes them co-resident.  All
// problems of one launch share the operand form and the run width P (a
// template parameter); the host groups them.
#include "dense_tc_persistent.cuh"
#include "internal.h"

#include <cstdlib>
#include <cstring>

namespace sbqa {

// One problem of a batched launch.
struct TbReq {
  TcMaps m;  // first, so that every map of every entry is 64-byte aligned
  StateView s;
  TpArgs a;
  StepTables t;
  int tile0;  // its first CTA
};

namespace {

template <int P, int OP, bool GEN>
__global__ void __launch_bounds__(kTpThreads, 1) k_solve_dense_tc_batched(const TbReq *__restrict__ q, int nq) {
  int r = 0;
  for (int k = 1; k < nq; ++k)
    if (int(blockIdx.x) >= q[k].tile0) r = k;
  const TbReq &d = q[r];
  if (threadIdx.x == 0) {  // the one thread that issues this CTA's TMA loads and stores
    tc::fence_tmap_acquire_sys(&d.m.A);
    tc::fence_tmap_acquire_sys(&d.m.B);
    tc::fence_tmap_acquire_sys(&d.m.Fst);
    if constexpr (OP == kOpBsb) {
      tc::fence_tmap_acquire_sys(&d.m.Bl);
      tc::fence_tmap_acquire_sys(&d.m.Fstl);
    } else {  // the views with several k-blocks per box
      tc::fence_tmap_acquire_sys(&d.m.A3);
      tc::fence_tmap_acquire_sys(&d.m.B3);
    }
  }
  const StateView s = d.s;
  const TpArgs a = d.a;
  const StepTables t = d.t;
  const int local = int(blockIdx.x) - d.tile0;
  solve_dense_tc_persistent<P, false, OP, GEN>(d.m, s, a, t, local / a.Ct, local % a.Ct);
}

#define SBQA_TB_PS(OP)                                                                                        \
  {{(const void *)k_solve_dense_tc_batched<1, OP, false>, (const void *)k_solve_dense_tc_batched<1, OP, false>},   \
   {(const void *)k_solve_dense_tc_batched<2, OP, false>, (const void *)k_solve_dense_tc_batched<2, OP, false>},   \
   {(const void *)k_solve_dense_tc_batched<4, OP, false>, (const void *)k_solve_dense_tc_batched<4, OP, true>},    \
   {(const void *)k_solve_dense_tc_batched<8, OP, false>, (const void *)k_solve_dense_tc_batched<8, OP, true>},    \
   {(const void *)k_solve_dense_tc_batched<16, OP, false>, (const void *)k_solve_dense_tc_batched<16, OP, true>},  \
   {(const void *)k_solve_dense_tc_batched<32, OP, false>, (const void *)k_solve_dense_tc_batched<32, OP, true>},  \
   {(const void *)k_solve_dense_tc_batched<64, OP, true>, (const void *)k_solve_dense_tc_batched<64, OP, true>},   \
   {(const void *)k_solve_dense_tc_batched<128, OP, true>, (const void *)k_solve_dense_tc_batched<128, OP, true>}}
// [operand form][log2 of the run width][GEN], as the single-problem solver's table
const void *const kTbFns[3][8][2] = {SBQA_TB_PS(kOpF8), SBQA_TB_PS(kOpBf16), SBQA_TB_PS(kOpBsb)};
#undef SBQA_TB_PS
const int kTbSmem[3] = {TpShape<false, kOpF8>::kSmem, TpShape<false, kOpBf16>::kSmem, TpShape<false, kOpBsb>::kSmem};

int log2_width(int P) {
  for (int q = 0; q < 8; ++q)
    if ((1 << q) == P) return q;
  return -1;
}

}  // namespace

struct TcBatch {
  int cap_reqs = 0, cap_tiles = 0;
  TbReq *host = nullptr;      // staging, 64-byte aligned
  TbReq *dev = nullptr;       // descriptor table
  uint32_t *flags = nullptr;  // step counters of all tiles of a launch
  int n = 0, tiles = 0, op = -1, P = 0, gen = 0;
};

cudaError_t tc_batch_create(TcBatch **out, int cap_reqs, int cap_tiles) {
  *out = nullptr;
  if (cap_reqs < 1 || cap_tiles < 1) return cudaErrorInvalidValue;
  TcBatch *b = new TcBatch;
  b->cap_reqs = cap_reqs;
  b->cap_tiles = cap_tiles;
  const size_t hb = (sizeof(TbReq) * size_t(cap_reqs) + 63) / 64 * 64;
  b->host = static_cast<TbReq *>(std::aligned_alloc(64, hb));
  cudaError_t e = b->host ? cudaSuccess : cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = cudaMalloc(&b->dev, sizeof(TbReq) * size_t(cap_reqs));
  if (e == cudaSuccess) e = cudaMalloc(&b->flags, sizeof(uint32_t) * size_t(cap_tiles));
  if (e != cudaSuccess) {
    tc_batch_destroy(b);
    return e;
  }
  *out = b;
  return cudaSuccess;
}

void tc_batch_destroy(TcBatch *b) {
  if (!b) return;
  std::free(b->host);
  if (b->dev) cudaFree(b->dev);
  if (b->flags) cudaFree(b->flags);
  delete b;
}

void tc_batch_clear(TcBatch *b) {
  b->n = b->tiles = 0;
  b->op = -1;
}

int tc_batch_tiles(const TcBatch *b) { return b->tiles; }
int tc_batch_size(const TcBatch *b) { return b->n; }

bool tc_batch_fits(const TcBatch *b, const void *plan, const StateView &s, int Kp) {
  const int tiles = (Kp / kTcBM) * (s.Cp / kTcBN);
  if (b->n >= b->cap_reqs || b->tiles + tiles > b->cap_tiles) return false;
  return b->n == 0 || (b->op == tc_op_of(plan) && b->P == s.P && b->gen == (s.Pr != s.P ? 1 : 0));
}

cudaError_t tc_batch_add(TcBatch *b, const void *plan, const StateView &s, int Kp, int *err, const float *h,
                         const StepTables &t, int n_begin, int n_end, int hold_step) {
  const int op = tc_op_of(plan);
  if (op < 0 || op > 2 || log2_width(s.P) < 0 || Kp % kTcBM != 0 || s.Cp % kTcBN != 0 || n_end < n_begin ||
      !tc_batch_fits(b, plan, s, Kp))
    return cudaErrorInvalidValue;
  TbReq &d = b->host[b->n];
  std::memcpy(&d.m, plan, sizeof(TcMaps));
  d.s = s;
  d.a = TpArgs{Kp, s.Cp / kTcBN, n_begin, n_end, err, h, b->flags + b->tiles, hold_step};
  d.t = t;
  d.tile0 = b->tiles;
  b->op = op;
  b->P = s.P;
  b->gen = s.Pr != s.P ? 1 : 0;
  b->tiles += (Kp / kTcBM) * (s.Cp / kTcBN);
  ++b->n;
  return cudaSuccess;
}

// Copies the descriptors (pageable staging: the call returns once the host
// buffer has been read, so the next batch may refill it), zeroes the flags and
// launches; every step of it is ordered on st behind the previous launch.
cudaError_t tc_batch_launch(TcBatch *b, cudaStream_t st) {
  if (b->n == 0) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(b->dev, b->host, sizeof(TbReq) * size_t(b->n), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->flags, 0, sizeof(uint32_t) * size_t(b->tiles), st);
  if (e != cudaSuccess) return e;
  const TbReq *q = b->dev;
  int nq = b->n;
  void *args[] = {&q, &nq};
  return cudaLaunchCooperativeKernel(kTbFns[b->op][log2_width(b->P)][b->gen], dim3(b->tiles), dim3(kTpThreads), args,
                                     kTbSmem[b->op], st);
}

cudaError_t tc_batch_set_attributes() {
  for (int op = 0; op < 3; ++op)
    for (int q = 0; q < 8; ++q)
      for (const void *f : kTbFns[op][q]) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kTbSmem[op]);
        if (e != cudaSuccess) return e;
      }
  return cudaSuccess;
}

int tc_batch_blocks() {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int op = 0; op < 3; ++op)
    for (int q = 0; q < 8; ++q)
      for (const void *f : kTbFns[op][q]) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kTpThreads, kTbSmem[op]) != cudaSuccess)
          return 0;
        best = per_sm < best ? per_sm : best;
      }
  return sms * best;
}

}  // namespace sbqa
