// tileset.h -- device view of a set of heterogeneous tiles (tile.cu).
#pragma once

#include <stdint.h>

struct sdd_tileset;

namespace sdd {

// Per-query tile statistics: T, R, absorbed weight, bubbles per ray, then the fractions of T
// and of R in kTileBins deflection-angle bins.
constexpr int kTileBins = 8;
constexpr int kTileStatCols = 4 + 2 * kTileBins;

struct TileSetDev {
  const float* heights;  // [n_tiles][(G+1)^2] thickness at the grid vertices
  const float* hmin;     // [n_tiles]
  const float* hmax;     // [n_tiles]
  const float* rho;      // [n_tiles] bubbles per cubic metre
  const float* d_mean;   // [n_tiles] mean thickness
  int n_tiles;
  int G;
  float L;
};

const TileSetDev* tileset_device_view(const sdd_tileset* t);

}  // namespace sdd
