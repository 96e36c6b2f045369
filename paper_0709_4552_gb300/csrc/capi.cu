// capi.cu -- the extern "C" entry points of libnbody (declared and
// documented in include/nbody.h): context lifetime, particle I/O, and the
// block-step sequence of Sec. 4.1 (select -> predict -> forces -> correct).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "nb_internal.cuh"

namespace {

constexpr double kDefaultEps = 1.0 / 256.0;        // Sec. 2: softening 2^-8
constexpr double kDefaultEta = 0.01;
constexpr double kDefaultDtMin = 1.0 / 4194304.0;  // Sec. 2: 2^-22
constexpr double kDefaultDtMax = 0.125;            // Sec. 2: 2^-3
// NB_LOOP_AUTO's crossovers (block-step loops timed per N on a GB300; the
// persistent mixed loop: 1.25x the host loop at N = 65536, 1.02x at 131072,
// 0.96x at 196608)
constexpr int64_t kAutoClusterMaxN = 2048;
constexpr int64_t kAutoPersistentMaxNMixed = 131072;
constexpr int64_t kAutoPersistentMaxNFp64 = 2048;
constexpr size_t kPinnedBytes = 1 << 16;
// largest block the on-the-fly j prediction takes under NB_JPREDICT_AUTO (the
// default): measured on a GB300 at N = 2^20, the in-kernel prediction costs
// ~5% of the force kernel at every block size, the separate predictor of all
// N a fixed ~0.095 ms, so the split wins below n ~ 1000 (n = 256: 1.13x of
// predict + forces; n = 1024: even; n = 4096: 0.96x)
constexpr int64_t kJpredictAutoMaxN = 1024;

int fail(nb_ctx* c, int code) {
  if (c && c->last_error == NB_OK && code != NB_OK) c->last_error = code;
  return code;
}

#define NB_CUDA(c, call)                                  \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) {                              \
      return fail((c), e_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA); \
    }                                                     \
  } while (0)

bool is_pow2(double x) {
  if (!(x > 0.0) || !isfinite(x)) return false;
  int e;
  return frexp(x, &e) == 0.5;
}

int select_device(nb_ctx* c) {
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return NB_ECUDA;
  if (cur != c->device && cudaSetDevice(c->device) != cudaSuccess) return NB_ECUDA;
  return NB_OK;
}

#define NB_ENTER(c)                              \
  do {                                           \
    if (!(c)) return NB_EINVAL;                  \
    if (select_device(c) != NB_OK) return fail((c), NB_ECUDA); \
  } while (0)

// entry points whose physics treats the j-store as ONE system
#define NB_SINGLE(c)                                             \
  do {                                                           \
    NB_ENTER(c);                                                 \
    if ((c)->n_clusters > 0) return fail((c), NB_ESTATE);        \
  } while (0)

void free_ctx(nb_ctx* c) {
  if (!c) return;
  void* dptrs[] = {c->m, c->x, c->v, c->a, c->jk, c->pot, c->t, c->dt, c->xp, c->vp, c->jA, c->jB,
                   c->jC, c->F, c->part, c->act, c->ident, c->ulist, c->sel_min, c->sel_cnt, c->red,
                   c->status, c->d_offsets, c->d_ceps, c->perm, c->iperm, c->skey[0], c->skey[1],
                   c->sval[0], c->sval[1], c->shist, c->tbox, c->mlist, c->pscratch, c->jm,
                   c->ext_x, c->ext_v, c->ext_A, c->ext_B, c->ext_C, c->ext_self, c->ext_ident, c->ext_gid};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  if (c->hpin) cudaFreeHost(c->hpin);
  for (int i = 0; i < 8; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  free(c->h_offsets);
  free(c->h_ceps);
  free(c);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, count * sizeof(T));
}

bool host_list_ok(const int32_t* l, int64_t n, int64_t N) {
  for (int64_t k = 0; k < n; ++k) {
    if (l[k] < 0 || l[k] >= N) return false;
    if (k > 0 && l[k - 1] >= l[k]) return false;
  }
  return true;
}

nb_tuning pick_tuning(const nb_ctx* c, int64_t n) {
  const nb_tuning& o = c->tune_override;
  if (o.ipt || o.threads || o.jtile || o.nsplit) {
    nb_tuning d = nb_default_tuning(c->precision);
    nb_tuning t{o.ipt ? o.ipt : d.ipt, o.threads ? o.threads : d.threads, o.jtile ? o.jtile : d.jtile,
                o.nsplit};
    if (nb_tuning_supported(c->precision, t)) return t;
  }
  const nb_tune_entry* e = nb_tune_find(c, NB_TUNE_SINGLE, c->n, n);
  if (e && nb_tuning_supported(c->precision, e->cfg)) return e->cfg;
  return nb_default_tuning(c->precision);
}

// device view of a caller's list (copied to ulist for host lists)
int stage_list(nb_ctx* c, const int32_t* list, int64_t n, int ptr_kind, const int32_t** d_list) {
  if (ptr_kind == NB_PTR_HOST) {
    if (!host_list_ok(list, n, c->n)) return fail(c, NB_EINVAL);
    NB_CUDA(c, cudaMemcpyAsync(c->ulist, list, n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
    *d_list = c->ulist;
  } else if (ptr_kind == NB_PTR_DEVICE) {
    NB_CUDA(c, nb_launch_check_list(list, n, c->n, &c->status->flags, c->stream));
    *d_list = list;
  } else {
    return fail(c, NB_EINVAL);
  }
  return NB_OK;
}

// copy a [count][3] AoS array into SoA rows dst[3][stride] at offset first
int put_vec(nb_ctx* c, const double* src, double* dst, int64_t first, int64_t count, int ptr_kind) {
  if (!src) {
    for (int k = 0; k < 3; ++k)
      NB_CUDA(c, cudaMemsetAsync(dst + k * c->n_pad + first, 0, count * sizeof(double), c->stream));
    return NB_OK;
  }
  const double* d_src = src;
  if (ptr_kind == NB_PTR_HOST) {
    NB_CUDA(c, cudaMemcpyAsync(c->part, src, 3 * count * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    d_src = c->part;
  }
  NB_CUDA(c, nb_launch_aos_to_soa(d_src, dst + first, count, c->n_pad, c->stream));
  return NB_OK;
}

int put_scalar(nb_ctx* c, const double* src, double* dst, int64_t first, int64_t count, int ptr_kind) {
  if (!src) {
    NB_CUDA(c, cudaMemsetAsync(dst + first, 0, count * sizeof(double), c->stream));
    return NB_OK;
  }
  NB_CUDA(c, cudaMemcpyAsync(dst + first, src, count * sizeof(double),
                             ptr_kind == NB_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                             c->stream));
  return NB_OK;
}

int get_vec(nb_ctx* c, const double* src_soa, int64_t stride, double* dst, int64_t count, int ptr_kind) {
  if (!dst) return NB_OK;
  if (ptr_kind == NB_PTR_HOST) {
    NB_CUDA(c, nb_launch_soa_to_aos(src_soa, stride, c->part, count, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(dst, c->part, 3 * count * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  } else {
    NB_CUDA(c, nb_launch_soa_to_aos(src_soa, stride, dst, count, c->stream));
  }
  return NB_OK;
}

int get_scalar(nb_ctx* c, const double* src, double* dst, int64_t count, int ptr_kind) {
  if (!dst) return NB_OK;
  NB_CUDA(c, cudaMemcpyAsync(dst, src, count * sizeof(double),
                             ptr_kind == NB_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                             c->stream));
  return NB_OK;
}

// particles [first, first + count) of a state array of `rows` rows to the
// caller (AoS for 3 rows); gathered through iperm in the resident order.
// Host copies are complete on return.
int get_rows(nb_ctx* c, const double* src, int rows, int64_t first, int64_t count, double* dst, int ptr_kind) {
  if (!dst) return NB_OK;
  int r;
  if (!c->perm_valid) {
    r = rows == 3 ? get_vec(c, src + first, c->n_pad, dst, count, ptr_kind)
                  : get_scalar(c, src + first, dst, count, ptr_kind);
  } else {
    NB_CUDA(c, nb_gather_rows(c, src, rows, first, count, ptr_kind == NB_PTR_HOST ? c->part : dst));
    r = NB_OK;
    if (ptr_kind == NB_PTR_HOST)
      NB_CUDA(c, cudaMemcpyAsync(dst, c->part, rows * count * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  if (r) return r;
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NB_OK;
}

// (re)compute the spatial order of the j-store when the particles changed or
// after sort_interval block steps; the next prediction writes that order
// (mixed path only: the FP64 path has no far-tile pass to gain from it)
int ensure_sorted(nb_ctx* c) {
  if (c->n_clusters > 0) return nb_ensemble_ensure_sorted(c);  // within each cluster
  if (c->n <= 0 || c->precision != NB_MIXED) return NB_OK;
  if (c->perm_valid && c->perm_age < c->sort_interval) return NB_OK;
  NB_CUDA(c, nb_spatial_sort(c));
  c->state_ver++;  // rows moved
  c->perm_valid = true;
  c->perm_age = 0;
  c->pred_valid = false;
  c->f_valid = false;
  return NB_OK;
}

// a caller's list on the device, as slots of the resident order
int caller_list(nb_ctx* c, const int32_t* list, int64_t n, int ptr_kind, const int32_t** d_slots) {
  if (ptr_kind == NB_PTR_DEVICE) {  // checked and mapped in one launch
    NB_CUDA(c, nb_check_map_to_slots(c, list, n, d_slots));
    return NB_OK;
  }
  const int32_t* d_list = nullptr;
  int r = stage_list(c, list, n, ptr_kind, &d_list);
  if (r) return r;
  NB_CUDA(c, nb_map_to_slots(c, d_list, n, d_slots));
  return NB_OK;
}

// block selection with the result copied to host: t_next, n
int select_block(nb_ctx* c, double* t_next, int64_t* n) {
  int rs = ensure_sorted(c);
  if (rs) return rs;
  NB_CUDA(c, nb_launch_select(c));
  unsigned char* h = (unsigned char*)c->hpin;
  NB_CUDA(c, cudaMemcpyAsync(h, c->sel_min + c->sel_ctas, 8, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaMemcpyAsync(h + 8, c->sel_cnt + c->sel_ctas, 4, cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  unsigned long long bits;
  int32_t cnt;
  memcpy(&bits, h, 8);
  memcpy(&cnt, h + 8, 4);
  double t;
  memcpy(&t, &bits, 8);
  *t_next = t;
  *n = cnt;
  return NB_OK;
}

float elapsed(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
    cudaGetLastError();  // do not leave the error for a later launch check to see
    return 0.0f;
  }
  return ms;
}

// blocks that take the on-the-fly j prediction (mixed single system)
bool use_jpredict(const nb_ctx* c, int64_t n) {
  return c->precision == NB_MIXED && c->n_clusters == 0 && n > 0 && n <= c->jpred_max_n;
}

// host side of the on-the-fly split: the list predicted to t and the far-test
// boxes of the j-memory tiles (null when the pass is off), one launch
int jm_host_side(nb_ctx* c, const int32_t* d_list, int64_t n, double t, const float4** boxes) {
  const bool b = c->perm_valid && c->far_tiles;
  NB_CUDA(c, nb_launch_jm_host_side(c, d_list, n, t, b));
  *boxes = b ? c->tbox : nullptr;
  return NB_OK;
}

// a correction of the rows d_list that keeps a current j-memory current (the
// corrector writes the corrected records), then counts the change of state
int correct_rows(nb_ctx* c, const int32_t* d_list, int64_t n, double t) {
  const bool keep = c->jm && c->jm_ver == c->state_ver;
  NB_CUDA(c, nb_launch_correct(c, d_list, n, t, keep));
  c->state_ver++;
  if (keep) c->jm_ver = c->state_ver;
  return NB_OK;
}

// one block step after selection (t_next, n known): predict, forces, correct
// (Sec. 4.1 steps 3-5); small blocks may take GRAPE's split instead (Sec. 4.4
// steps 3-7: the active particles predicted alone, the j on the fly)
int step_after_select(nb_ctx* c, double t, int64_t n) {
  const bool fused = use_jpredict(c, n);
  if (fused) {
    const int r = nb_jm_ensure(c);
    if (r) return fail(c, r);
  }
  NB_CUDA(c, cudaEventRecord(c->ev[0], c->stream));
  if (fused) {
    const float4* boxes = nullptr;
    int r = jm_host_side(c, c->act, n, t, &boxes);
    if (r) return r;
    NB_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    NB_CUDA(c, nb_forces_mixed_fused(c, c->act, n, pick_tuning(c, n), nullptr, t, boxes));
  } else {
    NB_CUDA(c, nb_launch_predict(c, t, false));
    NB_CUDA(c, cudaEventRecord(c->ev[1], c->stream));
    NB_CUDA(c, nb_forces(c, c->act, n));
  }
  NB_CUDA(c, cudaEventRecord(c->ev[2], c->stream));
  {
    const int r = correct_rows(c, c->act, n, t);
    if (r) return r;
  }
  NB_CUDA(c, cudaEventRecord(c->ev[3], c->stream));
  c->interactions += (double)n * (double)c->n;
  c->pred_valid = false;
  c->f_valid = false;
  c->ev_pending = true;
  c->steps += 1;
  c->perm_age += 1;
  return NB_OK;
}

void harvest_timings(nb_ctx* c) {
  if (!c->ev_pending) return;
  c->ev_pending = false;
  c->ms_pred += elapsed(c->ev[0], c->ev[1]);
  c->ms_force += elapsed(c->ev[1], c->ev[2]);
  c->ms_corr += elapsed(c->ev[2], c->ev[3]);
}

int device_status_code(nb_ctx* c, int64_t* underflows) {
  nb_dev_status st;
  NB_CUDA(c, cudaMemcpyAsync(c->hpin, c->status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  memcpy(&st, c->hpin, sizeof(st));
  if (underflows) *underflows = (int64_t)st.dt_underflows;
  if (st.flags & NB_ST_TIMEOUT) return NB_ETIMEOUT;
  if (st.flags & NB_ST_STALLED) return NB_ESTATE;  // (before NaNs: the stalled state's corrections make some)
  if (st.flags & NB_ST_NUMERIC) return NB_ENUMERIC;
  if (st.flags & NB_ST_BADLIST) return NB_EINVAL;
  return NB_OK;
}

// a force call's device outputs, written by the split reduction when there
// is one; they are cleared when the call returns, on every path
void set_device_outputs(nb_ctx* c, double* acc, double* jerk, double* pot, int ptr_kind) {
  const bool dev = ptr_kind == NB_PTR_DEVICE;
  c->fo_acc = dev ? acc : nullptr;
  c->fo_jerk = dev ? jerk : nullptr;
  c->fo_pot = dev ? pot : nullptr;
  c->fo_done = false;
}

struct DeviceOutputsScope {
  nb_ctx* c;
  ~DeviceOutputsScope() {
    c->fo_acc = c->fo_jerk = c->fo_pot = nullptr;
    c->fo_done = false;
  }
};

// the force rows of the last call to the caller (host copies complete on return)
int copy_forces_out(nb_ctx* c, int64_t n, double* acc, double* jerk, double* pot, int ptr_kind) {
  if (ptr_kind == NB_PTR_DEVICE) {  // one launch (none when the split reduction wrote them)
    const bool done = c->fo_done;
    c->fo_acc = c->fo_jerk = c->fo_pot = nullptr;
    c->fo_done = false;
    if (!done && (acc || jerk || pot)) NB_CUDA(c, nb_launch_forces_out(c, n, acc, jerk, pot, 0));
    return NB_OK;
  }
  int r;
  for (int q = 0; q < 2; ++q) {
    double* dst = q == 0 ? acc : jerk;
    if (!dst) continue;
    if ((r = get_vec(c, c->F + 3 * q * c->n_pad, c->n_pad, dst, n, ptr_kind))) return r;
    if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if ((r = get_scalar(c, c->F + 6 * c->n_pad, pot, n, ptr_kind))) return r;
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NB_OK;
}

}  // namespace

int nb_ensure_sorted(nb_ctx* c) { return ensure_sorted(c); }

// NB_LOOP_AUTO: the driver measured fastest per block step on this GPU for the
// context's precision and size (one N-body time unit of Plummer spheres): the
// cluster loop for the smallest mixed systems, the persistent loop while the
// block steps are latency-bound, the host loop beyond
static int auto_loop(nb_ctx* c) {
  if (c->precision == NB_MIXED && c->n <= kAutoClusterMaxN) {
    const int cs = nb_cluster_size(c);
    if (cs >= 1 && c->n <= (int64_t)cs * 1024) return NB_LOOP_CLUSTER;
  }
  if (c->n <= (c->precision == NB_MIXED ? kAutoPersistentMaxNMixed : kAutoPersistentMaxNFp64))
    return NB_LOOP_PERSISTENT;
  return NB_LOOP_HOST;
}

// the force dispatcher used by every entry point
cudaError_t nb_forces(nb_ctx* c, const int32_t* d_list, int64_t n) {
  const nb_tuning cfg = pick_tuning(c, n);
  if (c->precision == NB_FP64) return nb_forces_fp64(c, d_list, n, cfg);
  // mixed path in the resident spatial order: the block-selection list and
  // the identity list are ascending slots, i.e. already in that order; a
  // caller's list (mapped to slots) is visited sorted by slot.
  const int32_t* ord = nullptr;
  if (c->perm_valid && c->n_clusters == 0 && d_list != c->act && d_list != c->ident &&
      n >= 2048) {  // below that the sort costs more than the far tiles it finds
    cudaError_t e = nb_list_order(c, d_list, n, &ord);
    if (e != cudaSuccess) return e;
  }
  return nb_forces_mixed(c, d_list, n, cfg, ord);
}

extern "C" {

void nb_default_params(double* eps, double* eta, double* dt_min, double* dt_max) {
  if (eps) *eps = kDefaultEps;
  if (eta) *eta = kDefaultEta;
  if (dt_min) *dt_min = kDefaultDtMin;
  if (dt_max) *dt_max = kDefaultDtMax;
}

const char* nb_version(void) { return "libnbody 0.1 (sm_103a)"; }

const char* nb_strerror(int code) {
  switch (code) {
    case NB_OK: return "ok";
    case NB_EINVAL: return "invalid argument";
    case NB_ENOMEM: return "out of memory";
    case NB_ECUDA: return "CUDA runtime error";
    case NB_ENUMERIC: return "NaN or Inf in a result";
    case NB_EDTMIN: return "time-step criterion below dt_min";
    case NB_ETIMEOUT: return "bounded device wait timed out";
    case NB_ESTATE: return "call out of order";
    default: return "unknown status code";
  }
}

int nb_create(nb_ctx** out, int64_t n_max, int precision, int device, void* cuda_stream) {
  if (!out) return NB_EINVAL;
  *out = nullptr;
  if (n_max < 1 || n_max > ((int64_t)1 << 30) || (precision != NB_FP64 && precision != NB_MIXED))
    return NB_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return NB_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return NB_ECUDA;
  nb_ctx* c = (nb_ctx*)calloc(1, sizeof(nb_ctx));
  if (!c) return NB_ENOMEM;
  c->device = device;
  c->precision = precision;
  c->eps = kDefaultEps;
  c->eta = kDefaultEta;
  c->dt_min = kDefaultDtMin;
  c->dt_max = kDefaultDtMax;
  c->n_max = n_max;
  c->n_pad = ((n_max + NB_JPAD - 1) / NB_JPAD) * NB_JPAD;
  c->sel_ctas = 1024;
  c->sort_interval = 64;
  c->far_tiles = 1;
  c->jm_ver = -1;
  c->jpred_max_n = kJpredictAutoMaxN;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  c->sm_count = sms > 0 ? sms : 1;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    c->own_stream = true;
  }
  const size_t np = (size_t)c->n_pad;
  c->part_elems = 7 * std::max<int64_t>(c->n_pad, (int64_t)1 << 21);
#define NB_ALLOC(ptr, cnt) \
  if (e == cudaSuccess) e = dalloc(&(ptr), (cnt));
  NB_ALLOC(c->m, np) NB_ALLOC(c->x, 3 * np) NB_ALLOC(c->v, 3 * np) NB_ALLOC(c->a, 3 * np)
  NB_ALLOC(c->jk, 3 * np) NB_ALLOC(c->pot, np) NB_ALLOC(c->t, np) NB_ALLOC(c->dt, np)
  NB_ALLOC(c->xp, 3 * np) NB_ALLOC(c->vp, 3 * np) NB_ALLOC(c->jA, np) NB_ALLOC(c->jB, np)
  NB_ALLOC(c->jC, np) NB_ALLOC(c->F, 7 * np) NB_ALLOC(c->part, (size_t)c->part_elems)
  NB_ALLOC(c->act, np) NB_ALLOC(c->ident, np) NB_ALLOC(c->ulist, np) NB_ALLOC(c->mlist, np)
  NB_ALLOC(c->sel_min, (size_t)c->sel_ctas + 1) NB_ALLOC(c->sel_cnt, (size_t)c->sel_ctas + 1)
  NB_ALLOC(c->red, NB_RED_DOUBLES) NB_ALLOC(c->status, 1)
  NB_ALLOC(c->perm, np) NB_ALLOC(c->iperm, np) NB_ALLOC(c->skey[0], np) NB_ALLOC(c->skey[1], np)
  NB_ALLOC(c->sval[0], np) NB_ALLOC(c->sval[1], np) NB_ALLOC(c->shist, (np / 2048 + 1) * 256)
  NB_ALLOC(c->tbox, 2 * (np / NB_BOX_TILE + 1))
#undef NB_ALLOC
  if (e == cudaSuccess) e = cudaMallocHost(&c->hpin, kPinnedBytes);
  for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
  if (e == cudaSuccess) {
    // zero state, padding particles are written by the predictor
    const size_t bytes[] = {np, 3 * np, 3 * np, 3 * np, 3 * np, np, np, np};
    double* ptrs[] = {c->m, c->x, c->v, c->a, c->jk, c->pot, c->t, c->dt};
    for (int i = 0; i < 8 && e == cudaSuccess; ++i)
      e = cudaMemsetAsync(ptrs[i], 0, bytes[i] * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(nb_dev_status), c->stream);
    if (e == cudaSuccess) e = nb_launch_fill_ident(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess) {
    const int code = e == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA;
    free_ctx(c);
    cudaGetLastError();
    return code;
  }
  nb_tune_load_env(c);
  *out = c;
  return NB_OK;
}

void nb_destroy(nb_ctx* c) {
  if (!c) return;
  select_device(c);
  if (c->stream) cudaStreamSynchronize(c->stream);
  nb_ensemble_free(c);
  nb_persistent_free(c);
  nb_cluster_free(c);
  free_ctx(c);
}

int nb_set_params(nb_ctx* c, double eps, double eta, double dt_min, double dt_max) {
  if (!c) return NB_EINVAL;
  if (!(eps >= 0.0) || !isfinite(eps) || !(eta > 0.0) || !isfinite(eta) || !is_pow2(dt_min) ||
      !is_pow2(dt_max) || dt_min > dt_max)
    return fail(c, NB_EINVAL);
  c->eps = eps;
  c->eta = eta;
  c->dt_min = dt_min;
  c->dt_max = dt_max;
  return NB_OK;
}

int nb_get_params(nb_ctx* c, double* eps, double* eta, double* dt_min, double* dt_max) {
  if (!c) return NB_EINVAL;
  if (eps) *eps = c->eps;
  if (eta) *eta = c->eta;
  if (dt_min) *dt_min = c->dt_min;
  if (dt_max) *dt_max = c->dt_max;
  return NB_OK;
}

int nb_set_precision(nb_ctx* c, int precision) {
  if (!c) return NB_EINVAL;
  if (precision != NB_FP64 && precision != NB_MIXED) return fail(c, NB_EINVAL);
  if (precision != c->precision) c->pred_valid = false;
  c->precision = precision;
  return NB_OK;
}

int nb_set_j_particles(nb_ctx* c, int64_t first, int64_t count, const double* m, const double* x,
                       const double* v, const double* a, const double* jerk, const double* t,
                       const double* dt, int ptr_kind) {
  NB_ENTER(c);
  if (count < 0 || first < 0 || first + count > c->n_max || !m || !x || !v ||
      (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (count == 0) return NB_OK;
  NB_CUDA(c, nb_unsort(c));  // particle order while particles are written
  if (ptr_kind == NB_PTR_HOST) {
    const double* arrs[] = {m, x, v, a, jerk, t, dt};
    const int64_t lens[] = {count, 3 * count, 3 * count, 3 * count, 3 * count, count, count};
    for (int q = 0; q < 7; ++q) {
      if (!arrs[q]) continue;
      for (int64_t i = 0; i < lens[q]; ++i)
        if (!isfinite(arrs[q][i])) return fail(c, NB_EINVAL);
    }
  }
  int r;
  if ((r = put_scalar(c, m, c->m, first, count, ptr_kind))) return r;
  if ((r = put_vec(c, x, c->x, first, count, ptr_kind))) return r;
  if ((r = put_vec(c, v, c->v, first, count, ptr_kind))) return r;
  if ((r = put_vec(c, a, c->a, first, count, ptr_kind))) return r;
  if ((r = put_vec(c, jerk, c->jk, first, count, ptr_kind))) return r;
  if ((r = put_scalar(c, t, c->t, first, count, ptr_kind))) return r;
  if ((r = put_scalar(c, dt, c->dt, first, count, ptr_kind))) return r;
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  if (first + count > c->n) c->n = first + count;
  c->perm_valid = false;
  c->pred_valid = false;
  c->f_valid = false;
  c->plist_valid = false;
  c->state_ver++;
  return NB_OK;
}

int nb_set_n(nb_ctx* c, int64_t n) {
  if (!c) return NB_EINVAL;
  if (n < 0 || n > c->n_max) return fail(c, NB_EINVAL);
  if (select_device(c) != NB_OK) return fail(c, NB_ECUDA);
  NB_CUDA(c, nb_unsort(c));
  c->n = n;
  c->pred_valid = false;
  c->f_valid = false;
  c->plist_valid = false;
  c->perm_valid = false;
  c->state_ver++;
  return NB_OK;
}

int nb_get_n(nb_ctx* c, int64_t* n) {
  if (!c || !n) return NB_EINVAL;
  *n = c->n;
  return NB_OK;
}

int nb_get_particles(nb_ctx* c, int64_t first, int64_t count, double* m, double* x, double* v,
                     double* a, double* jerk, double* pot, double* t, double* dt, int ptr_kind) {
  NB_ENTER(c);
  if (count < 0 || first < 0 || first + count > c->n ||
      (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (count == 0) return NB_OK;
  int r;
  // one array at a time through the staging area
  const double* src[] = {c->x, c->v, c->a, c->jk, c->m, c->pot, c->t, c->dt};
  double* dst[] = {x, v, a, jerk, m, pot, t, dt};
  for (int q = 0; q < 8; ++q)
    if ((r = get_rows(c, src[q], q < 4 ? 3 : 1, first, count, dst[q], ptr_kind))) return r;
  return NB_OK;
}

int nb_next_block(nb_ctx* c, double* t_next, int32_t* active_idx, int64_t* n_active) {
  NB_SINGLE(c);
  if (!t_next || !n_active) return fail(c, NB_EINVAL);
  if (c->n <= 0) return fail(c, NB_ESTATE);
  int r = select_block(c, t_next, n_active);
  if (r) return r;
  if (active_idx && *n_active > 0) {
    // the device list holds slots of the resident order; the caller gets
    // ascending particle indices
    NB_CUDA(c, nb_map_to_particles(c, c->act, *n_active, c->ulist));
    NB_CUDA(c, cudaMemcpyAsync(active_idx, c->ulist, *n_active * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               c->stream));
    NB_CUDA(c, cudaStreamSynchronize(c->stream));
    std::sort(active_idx, active_idx + *n_active);
  }
  return NB_OK;
}

int nb_predict(nb_ctx* c, double t) {
  NB_SINGLE(c);
  if (c->n <= 0) return fail(c, NB_ESTATE);
  if (!isfinite(t)) return fail(c, NB_EINVAL);
  int rs = ensure_sorted(c);
  if (rs) return rs;
  NB_CUDA(c, nb_launch_predict(c, t, false));
  c->t_pred = t;
  c->pred_valid = true;
  c->plist_valid = false;
  return NB_OK;
}

int nb_compute_forces(nb_ctx* c, const int32_t* i_idx, int64_t n, double* acc, double* jerk, double* pot,
                      int ptr_kind) {
  NB_SINGLE(c);
  if (n < 0 || n > c->n || (n > 0 && !i_idx)) return fail(c, NB_EINVAL);
  if (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE) return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  if (!c->pred_valid) return fail(c, NB_ESTATE);
  const int32_t* d_list = nullptr;
  int r = caller_list(c, i_idx, n, ptr_kind, &d_list);
  if (r) return r;
  set_device_outputs(c, acc, jerk, pot, ptr_kind);
  const DeviceOutputsScope fo_scope{c};
  NB_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
  NB_CUDA(c, nb_forces(c, d_list, n));
  NB_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
  c->f_n = n;
  c->f_valid = true;
  c->f_list = d_list;
  c->plist_valid = false;
  c->interactions += (double)n * (double)c->n;
  r = copy_forces_out(c, n, acc, jerk, pot, ptr_kind);
  if (r) return r;
  if (ptr_kind == NB_PTR_HOST) c->ms_force += elapsed(c->ev[4], c->ev[5]);
  return NB_OK;
}

int nb_compute_forces_at(nb_ctx* c, double t, const int32_t* i_idx, int64_t n, double* acc, double* jerk,
                         double* pot, int ptr_kind) {
  NB_SINGLE(c);
  if (n < 0 || n > c->n || (n > 0 && !i_idx) || !isfinite(t)) return fail(c, NB_EINVAL);
  if (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE) return fail(c, NB_EINVAL);
  if (c->n <= 0) return fail(c, NB_ESTATE);
  if (n == 0) return NB_OK;
  int r = ensure_sorted(c);
  if (r) return r;
  const int32_t* d_list = nullptr;
  if ((r = caller_list(c, i_idx, n, ptr_kind, &d_list))) return r;
  set_device_outputs(c, acc, jerk, pot, ptr_kind);
  const DeviceOutputsScope fo_scope{c};
  NB_CUDA(c, cudaEventRecord(c->ev[4], c->stream));
  if (c->precision == NB_MIXED) {
    if ((r = nb_jm_ensure(c))) return fail(c, r);
    const float4* boxes = nullptr;
    if ((r = jm_host_side(c, d_list, n, t, &boxes))) return r;
    const int32_t* ord = nullptr;
    if (c->perm_valid && n >= 2048) NB_CUDA(c, nb_list_order(c, d_list, n, &ord));
    NB_CUDA(c, nb_forces_mixed_fused(c, d_list, n, pick_tuning(c, n), ord, t, boxes));
  } else {
    // the FP64 path predicts every particle (it has no on-the-fly prediction)
    NB_CUDA(c, nb_launch_predict(c, t, false));
    NB_CUDA(c, nb_forces(c, d_list, n));
  }
  NB_CUDA(c, cudaEventRecord(c->ev[5], c->stream));
  // the listed rows now hold their prediction at t, the others an older one
  c->pred_valid = c->precision == NB_FP64;
  c->t_pred = t;
  c->f_n = n;
  c->f_valid = true;
  c->f_list = d_list;
  c->plist_valid = true;
  c->t_plist = t;
  c->interactions += (double)n * (double)c->n;
  r = copy_forces_out(c, n, acc, jerk, pot, ptr_kind);
  if (r) return r;
  if (ptr_kind == NB_PTR_HOST) c->ms_force += elapsed(c->ev[4], c->ev[5]);
  return NB_OK;
}

int nb_set_jpredict(nb_ctx* c, int64_t max_n) {
  if (!c) return NB_EINVAL;
  if (max_n < NB_JPREDICT_AUTO) return fail(c, NB_EINVAL);
  c->jpred_max_n = max_n == NB_JPREDICT_AUTO ? kJpredictAutoMaxN : max_n;
  return NB_OK;
}

int nb_get_jpredict(nb_ctx* c, int64_t* max_n) {
  if (!c || !max_n) return NB_EINVAL;
  *max_n = c->jpred_max_n;
  return NB_OK;
}

// ---- particle and force exchange of the parallel algorithms (Sec. 4.2-4.3) ----

int nb_get_particles_idx(nb_ctx* c, const int32_t* idx, int64_t n, double* m, double* x, double* v, double* a,
                         double* jerk, double* pot, double* t, double* dt, int ptr_kind) {
  NB_ENTER(c);
  if (n < 0 || n > c->n || (n > 0 && !idx) || (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  const int32_t* slots = nullptr;
  int r = caller_list(c, idx, n, ptr_kind, &slots);
  if (r) return r;
  const double* src[] = {c->m, c->x, c->v, c->a, c->jk, c->pot, c->t, c->dt};
  double* dst[] = {m, x, v, a, jerk, pot, t, dt};
  const int rows[] = {1, 3, 3, 3, 3, 1, 1, 1};
  for (int q = 0; q < 8; ++q) {
    if (!dst[q]) continue;
    if (ptr_kind == NB_PTR_DEVICE) {
      NB_CUDA(c, nb_launch_gather_slots(c, slots, n, src[q], rows[q], dst[q]));
    } else {
      NB_CUDA(c, nb_launch_gather_slots(c, slots, n, src[q], rows[q], c->part));
      NB_CUDA(c, cudaMemcpyAsync(dst[q], c->part, rows[q] * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
  }
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NB_OK;
}

int nb_set_particles_idx(nb_ctx* c, const int32_t* idx, int64_t n, const double* m, const double* x,
                         const double* v, const double* a, const double* jerk, const double* pot, const double* t,
                         const double* dt, int ptr_kind) {
  NB_ENTER(c);
  if (n < 0 || n > c->n || (n > 0 && !idx) || (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  const double* src[] = {m, x, v, a, jerk, pot, t, dt};
  double* dst[] = {c->m, c->x, c->v, c->a, c->jk, c->pot, c->t, c->dt};
  const int rows[] = {1, 3, 3, 3, 3, 1, 1, 1};
  if (ptr_kind == NB_PTR_HOST)
    for (int q = 0; q < 8; ++q)
      if (src[q])
        for (int64_t i = 0; i < rows[q] * n; ++i)
          if (!isfinite(src[q][i])) return fail(c, NB_EINVAL);
  const int32_t* slots = nullptr;
  int r = caller_list(c, idx, n, ptr_kind, &slots);
  if (r) return r;
  for (int q = 0; q < 8; ++q) {
    if (!src[q]) continue;
    const double* s = src[q];
    if (ptr_kind == NB_PTR_HOST) {
      NB_CUDA(c, cudaMemcpyAsync(c->part, src[q], rows[q] * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      s = c->part;
    }
    NB_CUDA(c, nb_launch_scatter_slots(c, slots, n, s, rows[q], dst[q]));
  }
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->pred_valid = false;
  c->f_valid = false;
  c->plist_valid = false;
  c->state_ver++;
  return NB_OK;
}

int nb_get_predicted(nb_ctx* c, const int32_t* idx, int64_t n, double* xp, double* vp, int ptr_kind) {
  NB_SINGLE(c);
  if (n < 0 || n > c->n || (n > 0 && !idx) || (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  if (!c->pred_valid) return fail(c, NB_ESTATE);
  const int32_t* slots = nullptr;
  int r = caller_list(c, idx, n, ptr_kind, &slots);
  if (r) return r;
  const double* src[] = {c->xp, c->vp};
  double* dst[] = {xp, vp};
  for (int q = 0; q < 2; ++q) {
    if (!dst[q]) continue;
    if (ptr_kind == NB_PTR_DEVICE) {
      NB_CUDA(c, nb_launch_gather_slots(c, slots, n, src[q], 3, dst[q]));
    } else {
      NB_CUDA(c, nb_launch_gather_slots(c, slots, n, src[q], 3, c->part));
      NB_CUDA(c, cudaMemcpyAsync(dst[q], c->part, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
  }
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NB_OK;
}

int nb_forces_on(nb_ctx* c, int64_t n, const double* xi, const double* vi, const int64_t* gid, int64_t gid_base,
                 double* acc, double* jerk, double* pot, int accumulate, int ptr_kind) {
  NB_SINGLE(c);
  if (n < 0 || n > c->n_pad || (n > 0 && (!xi || !vi)) || (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  if (!c->pred_valid) return fail(c, NB_ESTATE);
  if (ptr_kind == NB_PTR_HOST)
    for (int64_t i = 0; i < 3 * n; ++i)
      if (!isfinite(xi[i]) || !isfinite(vi[i])) return fail(c, NB_EINVAL);
  NB_CUDA(c, nb_ext_reserve(c, n));
  const double* dx = xi;
  const double* dv = vi;
  const int64_t* dg = gid;
  if (ptr_kind == NB_PTR_HOST) {  // staged: the kernel below reads them before the force items reuse part
    NB_CUDA(c, cudaMemcpyAsync(c->part, xi, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    NB_CUDA(c, cudaMemcpyAsync(c->part + 3 * n, vi, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (gid) NB_CUDA(c, cudaMemcpyAsync(c->ext_gid, gid, n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    dx = c->part;
    dv = c->part + 3 * n;
    dg = gid ? c->ext_gid : nullptr;
  }
  NB_CUDA(c, nb_launch_ext_prepare(c, n, dx, dv, dg, gid_base));
  NB_CUDA(c, nb_forces_ext(c, n, pick_tuning(c, n)));
  c->f_valid = false;  // F holds the block's sums, not a list of this context
  c->interactions += (double)n * (double)c->n;
  if (ptr_kind == NB_PTR_DEVICE) {
    NB_CUDA(c, nb_launch_forces_out(c, n, acc, jerk, pot, accumulate));
    return NB_OK;
  }
  // host outputs through part: acc [0, 3n), jerk [3n, 6n), pot [6n, 7n)
  double* sa = acc ? c->part : nullptr;
  double* sj = jerk ? c->part + 3 * n : nullptr;
  double* sp = pot ? c->part + 6 * n : nullptr;
  if (accumulate) {
    if (sa) NB_CUDA(c, cudaMemcpyAsync(sa, acc, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (sj) NB_CUDA(c, cudaMemcpyAsync(sj, jerk, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (sp) NB_CUDA(c, cudaMemcpyAsync(sp, pot, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  NB_CUDA(c, nb_launch_forces_out(c, n, sa, sj, sp, accumulate));
  if (sa) NB_CUDA(c, cudaMemcpyAsync(acc, sa, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (sj) NB_CUDA(c, cudaMemcpyAsync(jerk, sj, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (sp) NB_CUDA(c, cudaMemcpyAsync(pot, sp, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NB_OK;
}

int nb_set_forces(nb_ctx* c, const int32_t* idx, int64_t n, const double* acc, const double* jerk,
                  const double* pot, int ptr_kind) {
  NB_SINGLE(c);
  if (n < 0 || n > c->n || (n > 0 && (!idx || !acc || !jerk || !pot)) ||
      (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE))
    return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  if (!c->pred_valid) return fail(c, NB_ESTATE);
  if (ptr_kind == NB_PTR_HOST)
    for (int64_t i = 0; i < n; ++i)
      if (!isfinite(acc[3 * i]) || !isfinite(acc[3 * i + 1]) || !isfinite(acc[3 * i + 2]) ||
          !isfinite(jerk[3 * i]) || !isfinite(jerk[3 * i + 1]) || !isfinite(jerk[3 * i + 2]) || !isfinite(pot[i]))
        return fail(c, NB_EINVAL);
  const int32_t* d_list = nullptr;
  int r = caller_list(c, idx, n, ptr_kind, &d_list);
  if (r) return r;
  if ((r = put_vec(c, acc, c->F, 0, n, ptr_kind))) return r;
  if ((r = put_vec(c, jerk, c->F + 3 * c->n_pad, 0, n, ptr_kind))) return r;
  if ((r = put_scalar(c, pot, c->F + 6 * c->n_pad, 0, n, ptr_kind))) return r;
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  c->f_n = n;
  c->f_valid = true;
  c->f_list = d_list;
  c->plist_valid = false;
  return NB_OK;
}

int nb_set_initial_forces(nb_ctx* c, const double* acc, const double* jerk, const double* pot, int ptr_kind) {
  NB_SINGLE(c);
  if (!acc || !jerk || !pot || (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE)) return fail(c, NB_EINVAL);
  const int64_t n = c->n;
  if (n <= 0) return fail(c, NB_ESTATE);
  if (ptr_kind == NB_PTR_HOST)
    for (int64_t i = 0; i < 3 * n; ++i)
      if (!isfinite(acc[i]) || !isfinite(jerk[i]) || (i < n && !isfinite(pot[i]))) return fail(c, NB_EINVAL);
  // particle order in, rows of the resident order out
  const int32_t* slots = c->perm_valid ? c->iperm : c->ident;
  const double* src[] = {acc, jerk, pot};
  double* dst[] = {c->F, c->F + 3 * c->n_pad, c->F + 6 * c->n_pad};
  const int rows[] = {3, 3, 1};
  for (int q = 0; q < 3; ++q) {
    const double* s = src[q];
    if (ptr_kind == NB_PTR_HOST) {
      NB_CUDA(c, cudaMemcpyAsync(c->part, src[q], rows[q] * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
      s = c->part;
    }
    NB_CUDA(c, nb_launch_scatter_slots(c, slots, n, s, rows[q], dst[q]));
  }
  NB_CUDA(c, nb_launch_initial_dt(c));
  c->pred_valid = false;
  c->f_valid = false;
  c->plist_valid = false;
  c->state_ver++;
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return device_status_code(c, nullptr) == NB_ENUMERIC ? fail(c, NB_ENUMERIC) : NB_OK;
}

int nb_correct(nb_ctx* c, const int32_t* i_idx, int64_t n, double t, int ptr_kind) {
  NB_SINGLE(c);
  if (n < 0 || n > c->n || (n > 0 && !i_idx) || !isfinite(t)) return fail(c, NB_EINVAL);
  if (n == 0) return NB_OK;
  // the listed particles must be predicted to t: by nb_predict, or by the
  // list prediction of nb_compute_forces_at
  const bool predicted = c->pred_valid || (c->plist_valid && t == c->t_plist);
  if (!c->f_valid || c->f_n != n || !predicted) return fail(c, NB_ESTATE);
  const int32_t* d_list = nullptr;
  int r = caller_list(c, i_idx, n, ptr_kind, &d_list);
  if (r) return r;
  if ((r = correct_rows(c, d_list, n, t))) return r;
  c->f_valid = false;
  c->pred_valid = false;
  c->plist_valid = false;
  if (ptr_kind == NB_PTR_HOST) NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return NB_OK;
}

int nb_initial_forces_and_dt(nb_ctx* c) {
  NB_ENTER(c);
  if (c->n_clusters > 0) {
    const int r = nb_ensemble_initial_forces_and_dt(c);
    return r == NB_OK ? r : fail(c, r);
  }
  if (c->n <= 0) return fail(c, NB_ESTATE);
  {
    int rs = ensure_sorted(c);
    if (rs) return rs;
  }
  NB_CUDA(c, nb_launch_predict(c, 0.0, true));
  NB_CUDA(c, nb_forces(c, c->ident, c->n));
  NB_CUDA(c, nb_launch_initial_dt(c));
  c->interactions += (double)c->n * (double)c->n;
  c->pred_valid = false;
  c->f_valid = false;
  c->plist_valid = false;
  c->state_ver++;
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  return device_status_code(c, nullptr) == NB_ENUMERIC ? fail(c, NB_ENUMERIC) : NB_OK;
}

int nb_step(nb_ctx* c, double* t_out, int64_t* n_out) {
  NB_SINGLE(c);
  if (c->n <= 0) return fail(c, NB_ESTATE);
  double t;
  int64_t n;
  int r = select_block(c, &t, &n);
  if (r) return r;
  if (!isfinite(t) || n <= 0) return fail(c, NB_ENUMERIC);
  if ((r = step_after_select(c, t, n))) return r;
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  harvest_timings(c);
  if (t_out) *t_out = t;
  if (n_out) *n_out = n;
  return NB_OK;
}

static int integrate_host_loop(nb_ctx* c, double t_end) {
  // block times strictly increase (every corrected particle moves on by at
  // least dt_min); a block time that does not is a state without valid steps
  // (e.g. never initialised: dt = 0), which would otherwise repeat forever
  double t_prev = -INFINITY;
  for (;;) {
    double t;
    int64_t n;
    int r = select_block(c, &t, &n);
    if (r) return r;
    harvest_timings(c);
    if (!isfinite(t) || n <= 0) return fail(c, NB_ENUMERIC);
    if (t > t_end) break;
    if (!(t > t_prev)) return fail(c, NB_ESTATE);
    t_prev = t;
    if ((r = step_after_select(c, t, n))) return r;
  }
  return NB_OK;
}

}  // extern "C"
int nb_integrate_graph(nb_ctx* c, double t_end);
extern "C" {

int nb_integrate(nb_ctx* c, double t_end, int loop) {
  NB_SINGLE(c);
  if (c->n <= 0) return fail(c, NB_ESTATE);
  if (!(t_end > 0.0) || !isfinite(t_end) || fmod(t_end, c->dt_max) != 0.0) return fail(c, NB_EINVAL);
  if (loop == NB_LOOP_AUTO) loop = auto_loop(c);
  if (loop != NB_LOOP_HOST && loop != NB_LOOP_GRAPH && loop != NB_LOOP_PERSISTENT && loop != NB_LOOP_CLUSTER)
    return fail(c, NB_EINVAL);  // (NB_LOOP_AUTO resolved above)
  if (loop == NB_LOOP_PERSISTENT && c->n > nb_persistent_max_n(c)) return fail(c, NB_EINVAL);
  if (loop == NB_LOOP_CLUSTER && (c->n > NB_CLUSTER_MAX_N || c->precision != NB_MIXED)) return fail(c, NB_EINVAL);
  int r = loop == NB_LOOP_GRAPH        ? nb_integrate_graph(c, t_end)
          : loop == NB_LOOP_PERSISTENT ? nb_integrate_persistent(c, t_end)
          : loop == NB_LOOP_CLUSTER    ? nb_integrate_cluster(c, t_end)
                                       : integrate_host_loop(c, t_end);
  if (loop != NB_LOOP_HOST) c->state_ver++;  // device-driven corrections (the host loop counts its own)
  c->plist_valid = false;
  if (r) return fail(c, r);
  r = device_status_code(c, nullptr);
  if (r == NB_ENUMERIC || r == NB_ETIMEOUT || r == NB_ESTATE) return fail(c, r);
  return NB_OK;
}

int nb_energy(nb_ctx* c, double* ekin, double* epot) {
  NB_SINGLE(c);
  if (c->n <= 0) return fail(c, NB_ESTATE);
  {
    int rs = ensure_sorted(c);
    if (rs) return rs;
  }
  NB_CUDA(c, nb_launch_predict(c, 0.0, true));
  NB_CUDA(c, nb_forces(c, c->ident, c->n));
  double* d_out = c->red + 2 * 1024;
  NB_CUDA(c, nb_launch_energy(c, c->F + 6 * c->n_pad, d_out));
  NB_CUDA(c, cudaMemcpyAsync(c->hpin, d_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  NB_CUDA(c, cudaStreamSynchronize(c->stream));
  double h[2];
  memcpy(h, c->hpin, sizeof(h));
  if (ekin) *ekin = h[0];
  if (epot) *epot = h[1];
  c->pred_valid = false;
  c->plist_valid = false;
  c->f_valid = false;
  return NB_OK;
}

int nb_get_timings(nb_ctx* c, double* ms_pred, double* ms_force, double* ms_corr, double* interactions,
                   int reset) {
  if (!c) return NB_EINVAL;
  if (ms_pred) *ms_pred = c->ms_pred;
  if (ms_force) *ms_force = c->ms_force;
  if (ms_corr) *ms_corr = c->ms_corr;
  if (interactions) *interactions = c->interactions;
  if (reset) c->ms_pred = c->ms_force = c->ms_corr = c->interactions = 0.0;
  return NB_OK;
}

int nb_get_counters(nb_ctx* c, int64_t* kernel_launches, int64_t* block_steps) {
  if (!c) return NB_EINVAL;
  if (kernel_launches) *kernel_launches = c->launches;
  if (block_steps) *block_steps = c->steps;
  return NB_OK;
}

int nb_check_device_status(nb_ctx* c, int64_t* dt_underflows) {
  NB_ENTER(c);
  return device_status_code(c, dt_underflows);
}

int nb_check_grid_barrier(nb_ctx* c, int phantom, double wait_ms) {
  NB_ENTER(c);
  if (!(wait_ms > 0.0) || !(wait_ms <= 4000.0)) return fail(c, NB_EINVAL);
  const int r = nb_persistent_barrier_check(c, phantom, wait_ms);
  return r == NB_OK ? r : fail(c, r);
}

int nb_last_error(nb_ctx* c) { return c ? c->last_error : NB_EINVAL; }

void nb_clear_error(nb_ctx* c) {
  if (!c) return;
  c->last_error = NB_OK;
  if (select_device(c) == NB_OK) {
    cudaMemsetAsync(c->status, 0, sizeof(nb_dev_status), c->stream);
    cudaStreamSynchronize(c->stream);
  }
}

int nb_set_tuning(nb_ctx* c, int i_per_thread, int threads, int j_tile, int n_split) {
  if (!c) return NB_EINVAL;
  nb_tuning t{i_per_thread, threads, j_tile, n_split};
  if (i_per_thread || threads || j_tile || n_split) {
    nb_tuning d = nb_default_tuning(c->precision);
    nb_tuning full{i_per_thread ? i_per_thread : d.ipt, threads ? threads : d.threads,
                   j_tile ? j_tile : d.jtile, n_split};
    if (!nb_tuning_supported(c->precision, full)) return fail(c, NB_EINVAL);
  }
  c->tune_override = t;
  return NB_OK;
}

int nb_set_far_tiles(nb_ctx* c, int enable) {
  if (!c) return NB_EINVAL;
  c->far_tiles = enable ? 1 : 0;
  return NB_OK;
}

int nb_get_far_tiles(nb_ctx* c, int* enabled) {
  if (!c || !enabled) return NB_EINVAL;
  *enabled = c->far_tiles;
  return NB_OK;
}

}  // extern "C"

namespace {

// the autotuner's search on the device slot list d_slots (n entries)
int autotune_on(nb_ctx* c, const int32_t* d_slots, int64_t n, int* i_per_thread, int* threads, int* j_tile,
                int* n_split) {
  static const int thr_list[] = {64, 128, 256};
  static const int ipt_mixed[] = {1, 2, 4};
  static const int jt_mixed[] = {64, 128, 256};
  static const int jt_fp64[] = {32, 64, 128};
  nb_tuning best{0, 0, 0, 0};
  float best_ms = 1e30f;
  const nb_tuning saved = c->tune_override;
  for (int ti = 0; ti < 3; ++ti) {
    for (int ii = 0; ii < (c->precision == NB_MIXED ? 3 : 1); ++ii) {
      for (int ji = 0; ji < 3; ++ji) {
        nb_tuning cfg{c->precision == NB_MIXED ? ipt_mixed[ii] : 1, thr_list[ti],
                      c->precision == NB_MIXED ? jt_mixed[ji] : jt_fp64[ji], 0};
        if (!nb_tuning_supported(c->precision, cfg)) continue;
        // the automatic split (0, sized from the kernel's occupancy), a
        // smaller and a larger explicit one, and (mixed) the splits that fill
        // exactly one and two waves of resident CTAs
        const int guess = nb_auto_split(c, n, cfg, 4);
        int splits[5] = {0, std::max(1, guess / 2), guess * 2, 0, 0};
        const int64_t itiles = (n + (int64_t)cfg.threads * cfg.ipt - 1) / ((int64_t)cfg.threads * cfg.ipt);
        const int per_sm = c->precision == NB_MIXED ? nb_mixed_ctas_per_sm(cfg) : 0;
        if (per_sm > 0 && guess > 1) {
          const int64_t R = (int64_t)c->sm_count * per_sm;
          for (int w = 1; w <= 2; ++w)
            if (w * R >= 2 * itiles) splits[2 + w] = (int)std::min<int64_t>(4096, w * R / itiles);
        }
        // explicit splits beyond the partial-sum scratch (or the supported
        // maximum) cannot launch: not candidates
        const int64_t cap = std::min<int64_t>(4096, c->part_elems / (7 * (((n + 31) / 32) * 32)));
        for (int si = 0; si < 5; ++si) {
          if (si > 0) {
            if (guess == 1 || splits[si] < 1 || splits[si] > cap) continue;
            bool seen = false;
            for (int sj = 1; sj < si; ++sj) seen = seen || splits[sj] == splits[si];
            if (seen) continue;
          }
          nb_tuning t = cfg;
          t.nsplit = splits[si];
          c->tune_override = t;
          NB_CUDA(c, nb_forces(c, d_slots, n));  // warm-up
          NB_CUDA(c, cudaEventRecord(c->ev[6], c->stream));
          NB_CUDA(c, nb_forces(c, d_slots, n));
          NB_CUDA(c, cudaEventRecord(c->ev[7], c->stream));
          NB_CUDA(c, cudaStreamSynchronize(c->stream));
          float ms = elapsed(c->ev[6], c->ev[7]);
          if (ms < 5.0f) {  // short launches: average a few more
            const int reps = 5;
            NB_CUDA(c, cudaEventRecord(c->ev[6], c->stream));
            for (int r = 0; r < reps; ++r) NB_CUDA(c, nb_forces(c, d_slots, n));
            NB_CUDA(c, cudaEventRecord(c->ev[7], c->stream));
            NB_CUDA(c, cudaStreamSynchronize(c->stream));
            ms = elapsed(c->ev[6], c->ev[7]) / reps;
          }
          if (ms < best_ms) {
            best_ms = ms;
            best = t;
          }
        }
      }
    }
  }
  c->tune_override = saved;
  c->f_valid = false;
  if (best.threads == 0) return fail(c, NB_ECUDA);
  // table entry for systems and blocks within a factor sqrt(2) of (N, n)
  nb_tune_store(c, NB_TUNE_SINGLE, c->n, n, best, best_ms);
  if (i_per_thread) *i_per_thread = best.ipt;
  if (threads) *threads = best.threads;
  if (j_tile) *j_tile = best.jtile;
  if (n_split) *n_split = best.nsplit;
  return NB_OK;
}

}  // namespace

extern "C" {

int nb_autotune(nb_ctx* c, int64_t n, int* i_per_thread, int* threads, int* j_tile, int* n_split) {
  NB_SINGLE(c);
  if (n < 1 || n > c->n) return fail(c, NB_EINVAL);
  if (!c->pred_valid) return fail(c, NB_ESTATE);
  return autotune_on(c, c->ident, n, i_per_thread, threads, j_tile, n_split);
}

int nb_autotune_list(nb_ctx* c, const int32_t* i_idx, int64_t n, int ptr_kind, int* i_per_thread, int* threads,
                     int* j_tile, int* n_split) {
  NB_SINGLE(c);
  if (n < 1 || n > c->n || !i_idx) return fail(c, NB_EINVAL);
  if (ptr_kind != NB_PTR_HOST && ptr_kind != NB_PTR_DEVICE) return fail(c, NB_EINVAL);
  if (!c->pred_valid) return fail(c, NB_ESTATE);
  const int32_t* d_slots = nullptr;
  const int r = caller_list(c, i_idx, n, ptr_kind, &d_slots);
  if (r) return r;
  return autotune_on(c, d_slots, n, i_per_thread, threads, j_tile, n_split);
}

}  // extern "C"
