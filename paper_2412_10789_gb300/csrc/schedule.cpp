// Tile list of the fused step over the relabelled rows (see the Schedule
// comment in gp_internal.h), the long-row chunk table, and the hub size.
#include <algorithm>
#include <vector>

#include "gp_internal.h"

namespace gp {

void build_schedule(Graph& g, const std::vector<int64_t>& rp) {
  const int64_t na = g.n_active;
  auto deg = [&](int64_t r) { return rp[r + 1] - rp[r]; };
  std::vector<int4> tiles;
  std::vector<int> poff(1, 0);
  auto push = [&](int64_t row, int64_t e0, uint32_t meta) {
    tiles.push_back(make_int4((int)row, (int)(uint32_t)(e0 & 0xffffffffLL), (int)(e0 >> 32), (int)meta));
  };
  // Long rows (more entries than a tile, or at least cfg.t_heavy): chunks of
  // kTileCap entries, whose partial sums the long-row kernel combines.
  const int64_t t_long = g.cfg.t_heavy > 0 ? std::min<int64_t>(g.cfg.t_heavy, kTileCap + 1) : kTileCap + 1;
  int64_t row = 0;
  while (row < na && deg(row) >= t_long) {
    const int64_t d = deg(row);
    const int64_t np = (d + kTileCap - 1) / kTileCap;
    if (np >= (int64_t(1) << 21)) throw Error{GP_ENOTSUP, "row too long for the chunk table"};
    for (int64_t p = 0; p < np; ++p) {
      const int64_t len = std::min<int64_t>(kTileCap, d - p * kTileCap);
      push(row, rp[row] + p * kTileCap, 1u | (uint32_t)(len << 1) | (uint32_t)(p << 11));
    }
    poff.push_back(poff.back() + (int)np);
    ++row;
  }
  const int nlong = (int)row;
  // Runs of rows with one equal degree d: tiles of up to kTileRows rows and
  // kTileCap entries, so entry e of a tile belongs to row row0 + (e - e0) / d.
  while (row < na) {
    const int64_t d = deg(row);
    int64_t end = row;
    while (end < na && deg(end) == d) ++end;
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(kTileRows, kTileCap / d));
    for (int64_t r = row; r < end; r += per) {
      const int64_t nr = std::min(per, end - r);
      push(r, rp[r], (uint32_t)(nr << 1) | (uint32_t)(d << 9));
    }
    row = end;
  }
  // shared-memory hub: as many leading rows of Q_k as fit beside the buffers
  int dev = 0, optin = 0;
  GP_CUDA_TRY(cudaGetDevice(&dev));
  GP_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int buffers = kStepWarps * kWarpSmemInts * (int)sizeof(int);
  const int reserve = 2048;  // static shared memory of the kernel
  int64_t hub = GP_HUB_CACHE ? std::max(0, (optin - buffers - reserve) / 4) : 0;
  hub = std::min<int64_t>(hub, na);
  hub = std::min<int64_t>(hub, g.n);
  hub &= ~int64_t(3);  // filled as float4
  Schedule& s = g.sched;
  s.ntiles = (int64_t)tiles.size();
  s.nlong = nlong;
  s.hub = (int)hub;
  s.smem_bytes = (int)(buffers + hub * 4);
  s.t_long = (int)t_long;
  Allocator* A = &g.alloc;
  s.tiles = (int4*)A->get(sizeof(int4) * std::max<size_t>(tiles.size(), 1));
  s.poff = (int*)A->get(sizeof(int) * poff.size());
  s.part = (float2*)A->get(sizeof(float2) * std::max(poff.back(), 1));
  if (!tiles.empty())
    GP_CUDA_TRY(cudaMemcpyAsync(s.tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                g.stream));
  GP_CUDA_TRY(cudaMemcpyAsync(s.poff, poff.data(), sizeof(int) * poff.size(), cudaMemcpyHostToDevice, g.stream));
  GP_CUDA_TRY(cudaStreamSynchronize(g.stream));
}

void free_schedule(Graph& g) {
  Schedule& s = g.sched;
  g.alloc.put(s.tiles);
  g.alloc.put(s.poff);
  g.alloc.put(s.part);
  s = Schedule{};
}

}  // namespace gp
