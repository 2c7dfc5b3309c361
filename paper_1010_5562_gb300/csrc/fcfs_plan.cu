// Plans: a call's sizes and launch-shape choices kept in an object.
//
// A plan records one workload (kind, total corners, clips, T, K, precision)
// and its knobs: the form of the contraction, the vertex splits, the tile shape
// and the batch unit size.  Knobs left automatic are resolved by the library's
// own rules when a call runs; a tuner sets them from measurements.  A plan's
// calls apply its knobs for their own duration on the calling thread, so plans
// never touch the process-wide test hooks and several plans can be used side
// by side.  Tiles of a layout are independent (Sec. III-A): the knobs change
// how the work is cut, never the result beyond FP32 rounding.
#include <new>

#include "fcfs_common.cuh"

namespace fcfs {
fcfs_status forward_plan_info(int64_t V, int32_t T, int32_t K, int32_t prec, int* form, int* splits, int* pair);
fcfs_status batch_plan_info(int64_t V, int32_t n, int32_t T, int32_t K, int32_t prec, int* grouped,
                            int* unit_chunks, int* pair);
}  // namespace fcfs

using namespace fcfs;

struct fcfs_plan_s {
  int32_t kind;
  int64_t V;
  int32_t n, T, K, prec;
  int64_t form;   // FCFS_KNOB_FORM value (-1 automatic)
  Knobs kn;
};

namespace {

// FCFS_KNOB_FORM of a plan -> Knobs::hybrid for its kind
int hybrid_of(int32_t kind, int64_t form) {
  if (form < 0) return -1;
  if (kind == FCFS_PLAN_BATCH) return form == 0 ? 0 : 2;   // direct units, or grouped
  return form == 0 ? 0 : (form == 1 ? 2 : 3);   // forward and adjoint: direct, grouped tc, grouped FFT
}

bool valid(const fcfs_plan_s* p) { return p != nullptr && p->kind >= 0 && p->kind <= FCFS_PLAN_ADJOINT; }

}  // namespace

extern "C" {

fcfs_status fcfs_plan_create(fcfs_plan* out, int32_t kind, int64_t V, int32_t n_clips, int32_t T, int32_t K,
                             int32_t prec) {
  if (!out) return FCFS_EINVAL;
  *out = nullptr;
  if (kind < FCFS_PLAN_FORWARD || kind > FCFS_PLAN_ADJOINT || V < 0) return FCFS_EINVAL;
  if (kind == FCFS_PLAN_BATCH ? n_clips < 1 : n_clips != 1) return FCFS_EINVAL;
  if (prec != FCFS_PREC_FP32 && prec != FCFS_PREC_SPLIT_F16) return FCFS_EINVAL;
  fcfs_plan_s* p = new (std::nothrow) fcfs_plan_s;
  if (!p) return FCFS_EINVAL;
  *p = fcfs_plan_s{kind, V, n_clips, T, K, prec, -1, Knobs{-1, 0, -1, 0}};
  // the sizes must be ones the entry points take
  if (fcfs_plan_workspace_size(p) == 0) {
    delete p;
    return FCFS_EUNSUPPORTED;
  }
  *out = p;
  return FCFS_OK;
}

void fcfs_plan_destroy(fcfs_plan plan) { delete plan; }

fcfs_status fcfs_plan_set(fcfs_plan p, int32_t knob, int64_t value) {
  if (!valid(p)) return FCFS_EINVAL;
  switch (knob) {
    case FCFS_KNOB_FORM:
      if (value < -1 || value > (p->kind == FCFS_PLAN_BATCH ? 1 : 2)) return FCFS_EINVAL;
      p->form = value;
      p->kn.hybrid = hybrid_of(p->kind, value);
      return FCFS_OK;
    case FCFS_KNOB_SPLITS:
      if (value < 0 || value > 4096 || p->kind != FCFS_PLAN_FORWARD) return FCFS_EINVAL;
      p->kn.splits = (int)value;
      return FCFS_OK;
    case FCFS_KNOB_PAIR:
      if (value < -1 || value > 1 || p->kind == FCFS_PLAN_ADJOINT) return FCFS_EINVAL;
      p->kn.pair = (int)value;
      return FCFS_OK;
    case FCFS_KNOB_UNIT_CHUNKS:
      if (value < 0 || value > 65536 || p->kind != FCFS_PLAN_BATCH) return FCFS_EINVAL;
      p->kn.unit_chunks = (int)value;
      return FCFS_OK;
  }
  return FCFS_EINVAL;
}

int64_t fcfs_plan_get(fcfs_plan p, int32_t knob) {
  if (!valid(p)) return -1;
  KnobScope ks(&p->kn);
  int form = 0, splits = 0, pair = 0, grouped = 0, chunks = 0;
  if (p->kind == FCFS_PLAN_FORWARD) {
    if (forward_plan_info(p->V, p->T, p->K, p->prec, &form, &splits, &pair) != FCFS_OK) return -1;
    switch (knob) {
      case FCFS_KNOB_FORM: return form;
      case FCFS_KNOB_SPLITS: return splits;
      case FCFS_KNOB_PAIR: return pair;
      case FCFS_KNOB_UNIT_CHUNKS: return 0;
    }
    return -1;
  }
  if (p->kind == FCFS_PLAN_BATCH) {
    if (batch_plan_info(p->V, p->n, p->T, p->K, p->prec, &grouped, &chunks, &pair) != FCFS_OK) return -1;
    switch (knob) {
      case FCFS_KNOB_FORM: return grouped;
      case FCFS_KNOB_SPLITS: return 0;
      case FCFS_KNOB_PAIR: return pair;
      case FCFS_KNOB_UNIT_CHUNKS: return chunks;
    }
    return -1;
  }
  if (knob == FCFS_KNOB_FORM) return fcfs_adjoint_grouped(p->V, p->T, p->K, p->prec);
  return knob == FCFS_KNOB_SPLITS || knob == FCFS_KNOB_PAIR || knob == FCFS_KNOB_UNIT_CHUNKS ? 0 : -1;
}

size_t fcfs_plan_workspace_size(fcfs_plan p) {
  if (!valid(p)) return 0;
  KnobScope ks(&p->kn);
  if (p->kind == FCFS_PLAN_FORWARD) return fcfs_workspace_size(p->V, p->T, p->K, p->prec);
  if (p->kind == FCFS_PLAN_BATCH) return fcfs_batch_workspace_size(p->V, p->n, p->T, p->K, p->prec);
  return fcfs_adjoint_workspace_size(p->V, p->T, p->K, p->prec);
}

fcfs_status fcfs_plan_forward(fcfs_plan p, const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                              uint32_t flags, float* F_out, int64_t* area_out, void* workspace, size_t ws_bytes,
                              void* stream) {
  if (!valid(p) || p->kind != FCFS_PLAN_FORWARD) return FCFS_EINVAL;
  KnobScope ks(&p->kn);
  return fcfs_forward(x, y, s, V, p->T, p->K, p->prec, flags, F_out, area_out, workspace, ws_bytes, stream);
}

fcfs_status fcfs_plan_batch(fcfs_plan p, const int32_t* x, const int32_t* y, const int8_t* s,
                            const int64_t* offsets, int64_t V_total, float* F_out, int64_t* area_out,
                            void* workspace, size_t ws_bytes, void* stream) {
  if (!valid(p) || p->kind != FCFS_PLAN_BATCH) return FCFS_EINVAL;
  KnobScope ks(&p->kn);
  return fcfs_batch(x, y, s, offsets, p->n, V_total, p->T, p->K, p->prec, 0u, F_out, area_out, workspace,
                    ws_bytes, stream);
}

fcfs_status fcfs_plan_adjoint(fcfs_plan p, const int32_t* x, const int32_t* y, const int8_t* s, int64_t V,
                              const float* dF, float* gx, float* gy, void* workspace, size_t ws_bytes,
                              void* stream) {
  if (!valid(p) || p->kind != FCFS_PLAN_ADJOINT) return FCFS_EINVAL;
  KnobScope ks(&p->kn);
  return fcfs_adjoint(x, y, s, V, p->T, p->K, p->prec, dF, gx, gy, workspace, ws_bytes, stream);
}

}  // extern "C"
