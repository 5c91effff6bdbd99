// pk_chain.cuh -- serial-chain robot constants as a kernel parameter.
//
// A serial chain is folded on the host (fold_chain) so that every fixed joint
// is merged into the next movable joint's origin and the fixed joints after
// the last movable joint form the tool transform; the result travels to the
// kernels by value (__grid_constant__), so every lane reads it from the
// constant bank.
#pragma once
#include "pk_internal.h"

namespace pk {

template <int N>
struct ChainC {
  float o_r[N][9];
  float o_t[N][3];
  float a[N][3];
  float tool_r[9], tool_t[3];
  float lo[N], hi[N], mid[N];
  uint32_t prism, orot, toolrot;
};

template <int N>
static ChainC<N> chain_const(const ChainHost& h) {
  ChainC<N> c;
  for (int j = 0; j < N; ++j) {
    for (int i = 0; i < 9; ++i) c.o_r[j][i] = h.o_r[j][i];
    for (int i = 0; i < 3; ++i) {
      c.o_t[j][i] = h.o_t[j][i];
      c.a[j][i] = h.a[j][i];
    }
    c.lo[j] = h.lo[j];
    c.hi[j] = h.hi[j];
    c.mid[j] = 0.5f * (h.lo[j] + h.hi[j]);
  }
  for (int i = 0; i < 9; ++i) c.tool_r[i] = h.tool_r[i];
  for (int i = 0; i < 3; ++i) c.tool_t[i] = h.tool_t[i];
  c.prism = h.prism;
  c.orot = h.orot;
  c.toolrot = h.toolrot;
  return c;
}

}  // namespace pk
