// Host side of the shared-memory ring streams (ring.cuh): which matrices
// qualify, the ring's geometry, and the kernels' shared-memory limit.
#include <map>
#include <mutex>
#include <utility>

#include "ring.cuh"

namespace amg {

RingGeom ring_plan(const Sell& M, int vbytes, int stages, const RingRows& rows) {
  RingGeom g;
  if (M.C != 32 || M.tpr != 1 || M.row0 || M.d16 || M.wmax <= 0 || M.nslices <= 0) return g;
  if (vbytes != 2 && vbytes != 4 && vbytes != 8) return g;
  if (stages == 0) stages = RING_DEFAULT_STAGES;
  if (stages < 2 || stages > RING_MAX_STAGES || rows.n > RING_MAX_ROWS) return g;
  for (int k = 0; k < rows.n; ++k) {
    if (rows.esz[k] != 4 && rows.esz[k] != 8) return g;
    if (((uintptr_t)rows.p[k] & 15u) != 0) return g;  // bulk copies start 16-byte aligned
  }
  auto up = [](size_t v) { return (v + 127) & ~(size_t)127; };
  // values, columns, per-row vectors; every block starts on 128 bytes
  size_t off = up((size_t)M.wmax * 32 * (size_t)vbytes);
  g.coff = (uint32_t)off;
  off = up(off + (size_t)M.wmax * 128);
  for (int k = 0; k < rows.n; ++k) {
    g.roff[k] = (uint32_t)off;
    off = up(off + 32 * (size_t)rows.esz[k]);
  }
  const size_t stage = off;
  const size_t tables = (size_t)RING_WARPS * RING_MAX_STAGES * (8 + 4);  // barriers, widths
  const size_t smem = (size_t)RING_WARPS * stages * stage + tables + RING_ALIGN_SLACK;
  if (smem > RING_SMEM_PER_CTA) return g;
  g.D = stages;
  g.stage = (uint32_t)stage;
  g.smem = smem;
  return g;
}

int ring_prepare(const void* fn, RingGeom& g, int64_t nslices, int num_sms) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, bool> attr;
  static std::map<std::pair<const void*, size_t>, int> occ;
  int dev = 0;
  AMG_CUDA_TRY(cudaGetDevice(&dev));
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    bool& done = attr[{fn, dev}];
    if (!done) {
      AMG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)RING_SMEM_PER_CTA));
      // the unified L1 / shared array mostly as shared memory: several rings per SM
      AMG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared));
      done = true;
    }
    int& nb = occ[{fn, g.smem}];  // the same on every device of one kind
    if (!nb) {
      AMG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, RING_THREADS,
                                                                 g.smem));
      if (nb < 1) nb = -1;
    }
    per_sm = nb;
  }
  if (per_sm < 1) return AMG_ERR_UNSUPPORTED;
  const int64_t need = (nslices + RING_WARPS - 1) / RING_WARPS;  // one slice per warp
  const int64_t full = (int64_t)num_sms * per_sm;
  g.grid = (int)(need < full ? need : full);
  return AMG_OK;
}

}  // namespace amg
