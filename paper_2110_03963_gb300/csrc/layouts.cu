// Host-only views of the tiled kernels' register layouts, read by CPU tests of their index maps:
// the tile index each thread register holds, its shared-memory slot, and where a tile index of
// block 0 sits in the state vector. The maps are the kernels' own constexpr functions (tj, spos,
// Geo::jthr / jreg, box_word), evaluated on the host.
#include "circ_impl.cuh"
#include "hc_kernels.cuh"

namespace {

template <int L>
void hc_layout(int32_t* index) {
  for (int tid = 0; tid < qvs::hc::NT; ++tid)
    for (int r = 0; r < qvs::hc::R; ++r) index[tid * qvs::hc::R + r] = qvs::hc::tj<L>(r, tid);
}

template <class G, int K>
void circ_layout(int32_t* index) {
  for (int tid = 0; tid < qvs::cf::NT; ++tid) {
    const int jt = G::template jthr<K>(tid);
    for (int r = 0; r < qvs::cf::R; ++r) index[tid * qvs::cf::R + r] = jt | G::jreg(K, r);
  }
}

template <class G>
int circ_geometry(int layout, int32_t* index, int* column_bits) {
  switch (layout) {
    case 0: circ_layout<G, 0>(index); break;
    case 1: circ_layout<G, 1>(index); break;
    case 2: circ_layout<G, 2>(index); break;
    default: return QVS_EINVAL;
  }
  *column_bits = qvs::cf::TB - G::B;
  return QVS_OK;
}

}  // namespace

extern "C" int qvs_tile_layout(int family, int log2n, int layout, int32_t* index, int32_t* slot, int32_t* global,
                               int* threads, int* regs, int* column_bits) {
  using namespace qvs;
  if (!index || !slot || !global || !threads || !regs || !column_bits) return QVS_EINVAL;
  if (family == QVS_LAYOUT_HYPERCUBE) {
    if (log2n != 0) return QVS_EINVAL;
    switch (layout) {
      case 0: hc_layout<0>(index); break;
      case 1: hc_layout<1>(index); break;
      case 2: hc_layout<2>(index); break;
      case 3: hc_layout<3>(index); break;
      default: return QVS_EINVAL;
    }
    for (int j = 0; j < hc::TILE; ++j) {
      slot[j] = hc::spos(j);
      global[j] = j;   // the contiguous tile type: tile index = index bits 0..11
    }
    *threads = hc::NT;
    *regs = hc::R;
    *column_bits = hc::TB;
    return QVS_OK;
  }
  using namespace qvs::cf;
  if (family == QVS_LAYOUT_CIRCULANT_ROW) {
    if (log2n != 0) return QVS_EINVAL;
    QVS_TRY(circ_geometry<GRow>(layout, index, column_bits));
    for (int j = 0; j < TILE; ++j) {
      slot[j] = cf::spos(j);
      global[j] = j;   // row tiles are contiguous
    }
    *threads = NT;
    *regs = R;
    return QVS_OK;
  }
  if (family == QVS_LAYOUT_CIRCULANT_BOX && (log2n != 26 || layout != 0)) return QVS_EINVAL;
  if (family != QVS_LAYOUT_CIRCULANT_COLUMN && family != QVS_LAYOUT_CIRCULANT_BOX) return QVS_EINVAL;
  int cb = 0, st = QVS_OK;
  switch (log2n) {
    case 17: st = circ_geometry<Geo<11, 1, 1, 1>>(layout, index, &cb); break;
    case 18: st = circ_geometry<Geo<10, 1, 1, 2>>(layout, index, &cb); break;
    case 19: st = circ_geometry<Geo<9, 1, 2, 2>>(layout, index, &cb); break;
    case 20: st = circ_geometry<Geo<8, 2, 2, 2>>(layout, index, &cb); break;
    case 21: st = circ_geometry<Geo<7, 2, 2, 3>>(layout, index, &cb); break;
    case 22: st = circ_geometry<Geo<6, 2, 3, 3>>(layout, index, &cb); break;
    case 23: st = circ_geometry<Geo<5, 3, 3, 3>>(layout, index, &cb); break;
    case 24: st = circ_geometry<Geo<4, 3, 3, 4>>(layout, index, &cb); break;
    case 25: st = circ_geometry<Geo<3, 3, 4, 4>>(layout, index, &cb); break;
    case 26: st = circ_geometry<Geo<2, 4, 4, 4>>(layout, index, &cb); break;
    case 27: st = circ_geometry<Geo<1, 4, 4, 5>>(layout, index, &cb); break;
    default: return QVS_EINVAL;
  }
  if (st != QVS_OK) return st;
  for (int j = 0; j < TILE; ++j) {
    // the transposes' slot, or for the tensor copy the word of the staged box
    slot[j] = family == QVS_LAYOUT_CIRCULANT_BOX ? box_word(j) : cf::spos(j);
    // block 0 of the column pass: the column bits stay low, the transform bits go above the 14
    // block bits
    global[j] = (j & ((1 << cb) - 1)) | ((j >> cb) << TB);
  }
  *threads = NT;
  *regs = R;
  *column_bits = cb;
  return QVS_OK;
}
