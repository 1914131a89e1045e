// Host check of the counting kernel's shared-memory layout (count_kernel.cuh:
// smem_layout, and the region offsets k_count derives from it): over every
// accumulation policy, home objects per lane, table and band size, slot
// count and histogram copies the planner can produce, each region -- the
// block's tables, and in each warp's block the count histogram, the second
// histogram or float-float columns, the queue, the two tile buffers, their
// weight tiles, the home box and the culled rows' index array -- starts on
// a 16-byte boundary, as cp.async rows and float4 loads need, and every
// warp's block is a multiple of 16 bytes.  It also checks that a tile
// buffer leaves room for the rows a culled run carries and pads (fewer
// than a step of 8 / HP rows on either side).
// Prints "layouts <n> misaligned <m>"; exits 1 on any misalignment.
//
// Build: nvcc -std=c++17 -I include -I <csrc> smem_layout_check.cu
#include "count_kernel.cuh"

#include <cstdio>

using namespace cute;

int main() {
  long n = 0, bad = 0;
  const int luts[] = {0, 1, 3, 100, 257, 8192, 8193};
  const int bands[] = {0, 1, 5, 77, 130};
  const int slots[] = {3, 33, 34, 42, 93, 95, 1764, 2704, 3000};
  const int copies[] = {1, 2, 4, 8, 16, 32};
  for (int lw : luts)
    for (int bw : bands)
      for (int ns : slots)
        for (int R : copies)
          for (int hp : {2, 4})
            for (int acc = 0; acc < 4; acc++)
              for (int wt = 0; wt < 2; wt++)
                for (int idx = 0; idx < 2; idx++) {
                  const SmemLayout L = smem_layout(lw, bw, ns, R, hp, acc, wt != 0, idx != 0);
                  // offsets as k_count takes them
                  const int whist = align16(ns * R * 4);
                  const int queue = L.hist_bytes, tiles = L.hist_bytes + L.queue_bytes;
                  const int wtiles = tiles + L.tile_bytes, box = wtiles + L.wtile_bytes;
                  const int cidx = box + 32, tile1 = tiles + kTileRows * 16;
                  const int offs[] = {L.lut_bytes, L.warp_bytes, whist, queue, tiles, tile1,
                                      wtiles, box, cidx};
                  bool ok = box + L.cull_bytes <= L.warp_bytes;
                  for (int o : offs) ok = ok && o % 16 == 0;
                  n++;
                  if (!ok) {
                    if (bad < 5)
                      std::printf("misaligned: lut %d band %d slots %d R %d hp %d acc %d wtile %d "
                                  "idx %d\n", lw, bw, ns, R, hp, acc, wt, idx);
                    bad++;
                  }
                }
  for (int hp : {2, 4}) {
    const int U = 8 / hp;
    if (!(U - 1 <= kTilePre && U - 1 <= kTileRows - kTilePre - kTile)) bad++;
  }
  std::printf("layouts %ld misaligned %ld\n", n, bad);
  return bad ? 1 : 0;
}
