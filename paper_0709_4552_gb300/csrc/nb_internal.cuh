// nb_internal.cuh -- context layout and kernel launchers shared by the
// translation units of libnbody (the GB300 direct-sum Hermite engine).
//
// HBM layout of one context (n_max particles, n_pad = n_max rounded up to
// NB_JPAD so that every j-tile is full; padding particles have m = 0 and sit
// far away, so they contribute exactly zero):
//
//   master state, FP64 structure-of-arrays (component-major):
//     m[n_pad], x[3][n_pad], v[3][n_pad], a[3][n_pad], jk[3][n_pad],
//     pot[n_pad], t[n_pad], dt[n_pad]                        128 B/particle
//   predicted j-particles (predictor output, Sec. 4.1 step 3):
//     FP64 path:  xp[3][n_pad], vp[3][n_pad]                  48 B/particle
//     mixed path: jA[n_pad] = float4(x_hi, y_hi, z_hi, m)
//                 jB[n_pad] = float4(x_lo, y_lo, z_lo, vx)
//                 jC[n_pad] = float2(vy, vz)                    40 B/particle
//   force results of the last call, by position k in the active list:
//     F[7][n_pad] = (ax, ay, az, jx, jy, jz, pot), FP64        56 B/particle
//   split-j partial sums: part[n_split][7][n_i]                (bounded)
//   active list: act[n_pad] (int32, ascending), identity list ident[n_pad]
//
// Resident order: in the mixed path every per-particle array above is stored
// in the spatial (Morton) order of the particles once it has been computed
// (perm_valid): row s holds particle perm[s].  Every kernel works on rows
// ("slots"); particle indices exist only at the C ABI, which maps caller
// lists through iperm and returns particles through perm.  The arrays keep
// their addresses when the order changes (the permutation goes through a
// scratch block and back), so captured CUDA graphs stay valid.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nbody.h"

#define NB_JPAD 1024          // j-store padding granule (max j-tile)
#define NB_PAD_POS 1.0e15     // position of padding particles (m = 0)
#define NB_BOX_TILE 128       // j-tile of the spatial boxes (the mixed default j-tile)
#define NB_RED_DOUBLES (8192 + 16)  // reduction scratch: partials, energies, bounding box
#define NB_BBOX_OFFSET 8192         // 6 doubles of the particles' bounding box

// device status word bits
#define NB_ST_NUMERIC 1u
#define NB_ST_TIMEOUT 2u
#define NB_ST_BADLIST 4u
#define NB_ST_STALLED 8u   // a device-driven loop's block time stopped increasing (no valid steps)

struct nb_dev_status {
  unsigned int flags;          // NB_ST_* bits, sticky until cleared
  unsigned int pad;
  unsigned long long dt_underflows;
};

struct nb_tuning {
  int ipt;      // i-particles per thread
  int threads;  // threads per CTA (batched items: the i-tile)
  int jtile;    // j-particles per shared-memory tile
  int nsplit;   // split-j factor (0 = automatic)
  int waves;    // batched items: force items planned per resident CTA (0 = default)
};

// the autotuner's table (tune.cu): the fastest measured launch per workload bin
#define NB_TUNE_SINGLE 0   // force launch of the host-driven path, bins of (N, n)
#define NB_TUNE_BATCHED 1  // items of the device-driven loops, bins of (median N_c, clusters C)
#define NB_TUNE_MAX 64
struct nb_tune_entry {
  int kind;             // NB_TUNE_SINGLE / NB_TUNE_BATCHED
  int precision;
  int64_t N_lo, N_hi;   // N (single) or median cluster size (batched), [lo, hi)
  int64_t n_lo, n_hi;   // active block n (single) or cluster count C (batched), [lo, hi)
  nb_tuning cfg;
  double ms;            // measured time of cfg when it was chosen
};

struct nb_ctx {
  int device;
  int precision;
  int sm_count;
  cudaStream_t stream;
  bool own_stream;
  int64_t n_max, n_pad, n;
  double eps, eta, dt_min, dt_max;
  int last_error;

  // master state
  double *m, *x, *v, *a, *jk, *pot, *t, *dt;
  // predicted
  double *xp, *vp;
  float4 *jA, *jB;
  float2 *jC;
  double t_pred;         // time of the last prediction
  bool pred_valid;
  // forces of the last call
  double* F;             // [7][n_pad]
  int64_t f_n;           // size of the list of the last force call
  bool f_valid;
  const int32_t* f_list; // device list the forces belong to (act / ident / user copy)
  // split-j scratch
  double* part;
  int64_t part_elems;    // capacity in doubles
  // lists
  int32_t *act, *ident, *ulist;   // ulist: device copy of a caller's host list
  // block selection scratch
  unsigned long long* sel_min;  // per-CTA minima [sel_ctas] + result at [sel_ctas]
  int32_t* sel_cnt;             // per-CTA counts [sel_ctas] + total at [sel_ctas]
  int sel_ctas;
  double* red;                  // reduction scratch [NB_RED_DOUBLES]
  // resident spatial (Morton) order of the particle arrays (spatial.cu)
  int32_t *perm, *iperm;        // perm[slot] = particle, iperm[particle] = slot
  int32_t* mlist;               // a caller's list mapped to slots
  double* pscratch;             // 16 x n_pad doubles for reordering (allocated on first use)
  uint32_t* skey[2];            // radix-sort key buffers
  int32_t* sval[2];             // radix-sort value buffers
  int32_t* shist;               // radix-sort digit histograms
  float4* tbox;                 // per j-tile box: (lo, rmax), (hi, 0)
  bool perm_valid;              // the arrays are in the order perm (else slot = particle)
  int perm_age;                 // block steps since the last sort
  int sort_interval;            // re-sort after this many block steps
  // device status
  nb_dev_status* status;
  // pinned host staging for small results
  void* hpin;
  // timings
  cudaEvent_t ev[8];
  double ms_pred, ms_force, ms_corr, interactions;
  bool ev_pending;           // step events recorded but not yet read
  int64_t launches;          // kernels launched by this context (all launchers)
  int64_t steps;             // block steps taken
  // mixed path: hi-only differences on (warp, j-tile) pairs that pass the
  // far test (1, the default), or double-single differences everywhere (0)
  int far_tiles;
  // on-the-fly j prediction (GRAPE's split of Sec. 4.4 steps 3-4, onboard.cu):
  // the j-memory records jm[5][n_pad] (allocated on first use), valid while
  // jm_ver == state_ver (every change of the particle state bumps state_ver);
  // host-loop blocks of n <= jpred_max_n take the fused path
  float4* jm;
  int64_t state_ver, jm_ver;
  int64_t jpred_max_n;
  bool plist_valid;          // the last force call predicted its own list (nb_compute_forces_at)
  double t_plist;
  // i-particles held elsewhere (the ring algorithm's visiting block, exchange.cu),
  // capacity ext_cap, allocated on first use
  double *ext_x, *ext_v;     // SoA [3][ext_cap]
  float4 *ext_A, *ext_B;
  float2* ext_C;
  int32_t *ext_self, *ext_ident;
  int64_t* ext_gid;          // staged global ids of a host block
  int64_t ext_cap;
  // a caller's device outputs of the current force call (AoS acc, jerk and
  // pot, any NULL): the split reduction writes them beside F and sets fo_done
  double *fo_acc, *fo_jerk, *fo_pot;
  bool fo_done;
  // tuning
  nb_tuning tune_override;   // all-zero = automatic
  nb_tune_entry tune_table[NB_TUNE_MAX];
  int tune_count;

  // ensemble
  int32_t n_clusters;
  int64_t* d_offsets;   // [n_clusters + 1]
  double* d_ceps;       // [n_clusters]
  int64_t* h_offsets;
  double* h_ceps;
  void* ens;            // ensemble work area (ensemble.cu)
  void* loop;           // persistent-loop work area (persistent.cu)
  void* cloop;          // cluster-loop work area (cluster.cu)
};

// ---- launchers (integrator.cu) -------------------------------------------
cudaError_t nb_launch_predict(nb_ctx* c, double t, bool own_time);
cudaError_t nb_launch_select(nb_ctx* c);    // writes act, sel_cnt[total], sel_min[result]
// write_jm: also write the corrected rows' j-memory records (c->jm)
cudaError_t nb_launch_correct(nb_ctx* c, const int32_t* d_list, int64_t n, double t, bool write_jm = false);
cudaError_t nb_launch_initial_dt(nb_ctx* c);
cudaError_t nb_launch_energy(nb_ctx* c, const double* d_pot, double* d_out2);
cudaError_t nb_launch_fill_ident(nb_ctx* c);
cudaError_t nb_launch_aos_to_soa(const double* src, double* dst, int64_t count, int64_t stride_dst,
                                 cudaStream_t s);
cudaError_t nb_launch_soa_to_aos(const double* src, int64_t stride_src, double* dst, int64_t count,
                                 cudaStream_t s);
cudaError_t nb_launch_check_list(const int32_t* d_list, int64_t n, int64_t N, unsigned int* d_flag,
                                 cudaStream_t s);

// ---- on-the-fly j prediction (onboard.cu) -----------------------------------
// j-memory records of the rows in d_list[0..count) (d_list NULL: every row
// [0, n_pad), padding rows included) from the FP64 state
cudaError_t nb_launch_jm_write(nb_ctx* c, const int32_t* d_list, int64_t count);
// one launch: the listed rows predicted to t (FP64 xp, vp and the mixed
// jA/jB/jC rows) and, with boxes, the far-test boxes of the 128-row tiles
// from the j-memory, grown by each particle's reach (into c->tbox)
cudaError_t nb_launch_jm_host_side(nb_ctx* c, const int32_t* d_list, int64_t n, double t, bool boxes);
// make the j-memory current (allocate, rebuild when the state changed)
int nb_jm_ensure(nb_ctx* c);

// ---- exchange between ranks (exchange.cu) ----------------------------------
// dst[k][r] = src[r][slots[k]] (rows 1 or 3) and the reverse
cudaError_t nb_launch_gather_slots(nb_ctx* c, const int32_t* slots, int64_t n, const double* src, int rows,
                                   double* dst);
cudaError_t nb_launch_scatter_slots(nb_ctx* c, const int32_t* slots, int64_t n, const double* src, int rows,
                                    double* dst);
cudaError_t nb_ext_reserve(nb_ctx* c, int64_t n);  // i-arrays for n particles held elsewhere
// the block (device AoS xi, vi [n][3]; gid nullable) into the i-arrays
cudaError_t nb_launch_ext_prepare(nb_ctx* c, int64_t n, const double* xi, const double* vi, const int64_t* gid,
                                  int64_t base);
cudaError_t nb_forces_ext(nb_ctx* c, int64_t n, const nb_tuning& cfg);  // forces on the i-arrays -> F
// F rows [0, n) to device outputs (any NULL), added on when accumulate
cudaError_t nb_launch_forces_out(nb_ctx* c, int64_t n, double* acc, double* jerk, double* pot, int accumulate);

// ---- launchers (force_fp64.cu / force_mixed.cu) ----------------------------
namespace nbk {
struct ISrc;  // i-particles held elsewhere (force_common.cuh)
}
// forces on the list d_list[0..n) from all N j; results to c->F.  isrc
// (optional): the i-particles come from those arrays instead of the j-store
cudaError_t nb_forces_fp64(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg,
                           const nbk::ISrc* isrc = nullptr);
// ord (optional): processing order of the list positions (spatial order)
cudaError_t nb_forces_mixed(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg,
                            const int32_t* ord = nullptr, const nbk::ISrc* isrc = nullptr);
// the mixed item with the j-tiles predicted to T from the j-memory
cudaError_t nb_forces_mixed_fused(nb_ctx* c, const int32_t* d_list, int64_t n, const nb_tuning& cfg,
                                  const int32_t* ord, double T, const float4* boxes);
// split-j reduction (force_fp64.cu): part[S][7][n] -> F in fixed order, potential sign
cudaError_t nb_launch_split_reduce(nb_ctx* c, const int32_t* d_list, int64_t n, int nsplit,
                                   int64_t stride);
// the same for double-single partials (float2 in each 8-byte slot, force_mixed.cu),
// summed in FP32; also writes the caller's device outputs c->fo_* when set
cudaError_t nb_launch_split_reduce_ds(nb_ctx* c, int64_t n, int nsplit, int64_t stride);
bool nb_tuning_supported(int precision, const nb_tuning& cfg);
nb_tuning nb_default_tuning(int precision);
// resident CTAs per SM of the mixed launch of shape cfg (0 = unsupported)
int nb_mixed_ctas_per_sm(const nb_tuning& cfg);
// split-j factor for a kernel with per_sm resident CTAs per SM
int nb_auto_split(const nb_ctx* c, int64_t n, const nb_tuning& cfg, int per_sm);

// the force dispatcher (capi.cu): picks the tuning and precision path
cudaError_t nb_forces(nb_ctx* c, const int32_t* d_list, int64_t n);

// spatial.cu
cudaError_t nb_spatial_sort(nb_ctx* c);       // new resident order from the current positions
// new resident order: rows stably sorted by skey[0] (low `bits` bits), sval[0] = row numbers
cudaError_t nb_order_rows_by_keys(nb_ctx* c, int bits);
cudaError_t nb_unsort(nb_ctx* c);             // back to particle order (perm_valid = false)
// caller list of particles -> list of slots in c->mlist (*out = d_list when unsorted)
cudaError_t nb_map_to_slots(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** out);
// a caller's device list checked (ascending, in [0, N): else NB_ST_BADLIST) and
// mapped to slots in one launch (*out = c->mlist, or d_list when unsorted)
cudaError_t nb_check_map_to_slots(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** out);
// slots -> particles: out[k] = perm[in[k]] (in == out allowed)
cudaError_t nb_map_to_particles(nb_ctx* c, const int32_t* in, int64_t n, int32_t* out);
// rows of particles [first, first + count) of a state array (rows x n_pad) to AoS dst
cudaError_t nb_gather_rows(nb_ctx* c, const double* src, int rows, int64_t first, int64_t count, double* dst);
cudaError_t nb_launch_tile_boxes(nb_ctx* c);  // tbox from the predicted (permuted) j-store
// processing order of a list of slots: positions sorted by slot (device array of n positions)
cudaError_t nb_list_order(nb_ctx* c, const int32_t* d_list, int64_t n, const int32_t** ord);

// tune.cu: the autotuner's table
// the entry of kind for (N, n) and the context's precision, or null
const nb_tune_entry* nb_tune_find(const nb_ctx* c, int kind, int64_t N, int64_t n);
// record cfg for the bin around (N, n) (replaces an overlapping entry)
void nb_tune_store(nb_ctx* c, int kind, int64_t N, int64_t n, const nb_tuning& cfg, double ms);
// the table of the file named by NB_TUNE_FILE, if that is set (errors ignored)
void nb_tune_load_env(nb_ctx* c);

// capi.cu: (re)compute the resident spatial order when it is due (mixed path)
int nb_ensure_sorted(nb_ctx* c);

// ensemble.cu
void nb_ensemble_free(nb_ctx* c);
// (re)compute the spatial order within each cluster when it is due (mixed ensembles)
int nb_ensemble_ensure_sorted(nb_ctx* c);
int nb_integrate_graph(nb_ctx* c, double t_end);

// cluster.cu: the block-step loop of one small mixed system on one thread-block cluster
int nb_integrate_cluster(nb_ctx* c, double t_end);
void nb_cluster_free(nb_ctx* c);
int nb_cluster_size(nb_ctx* c);  // CTAs per cluster the GPU co-schedules (16, 8, or 0)

// persistent.cu: the block-step loop of one system as one cooperative launch
int nb_integrate_persistent(nb_ctx* c, double t_end);
void nb_persistent_free(nb_ctx* c);
// largest N the loop takes at the context's precision (a full-block force
// phase stays far inside the barrier wait)
inline int64_t nb_persistent_max_n(const nb_ctx* c) {
  return c->precision == NB_MIXED ? NB_PERSISTENT_MAX_N : NB_PERSISTENT_MAX_N_FP64;
}
// the grid barrier's bounded wait (phantom: wait for one CTA more than launched)
int nb_persistent_barrier_check(nb_ctx* c, int phantom, double wait_ms);

// ---- device helpers ---------------------------------------------------------
// the low 10 bits of a moved to every third bit (one axis of a Morton code)
__device__ __forceinline__ uint32_t nb_spread10(uint32_t a) {
  a &= 0x3FFu;
  a = (a | (a << 16)) & 0x030000FFu;
  a = (a | (a << 8)) & 0x0300F00Fu;
  a = (a | (a << 4)) & 0x030C30C3u;
  a = (a | (a << 2)) & 0x09249249u;
  return a;
}

__device__ __forceinline__ float nb_rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) in FP64 for any x >= 0.  For x in the FP32 normal range
// [2^-126, 2^128) the FP32 hardware seed is refined by one 2nd-order
// Newton-Raphson (Householder) step,
//   e = 1 - x y0^2,  y = y0 (1 + e/2 + 3 e^2 / 8),
// whose relative error is O(e^3) ~ 2^-63 for |e| <= 2^-21.  Outside that
// range the seed is 0 or Inf (the FP32 conversion overflows, or underflows
// and is flushed), and CUDA's double-precision rsqrt takes over: x = 0 gives
// +Inf, x = Inf gives 0, tiny and huge finite x their correctly scaled
// values.  The test costs two FP32 compares per call, off the FP64 pipe.
__device__ __forceinline__ double nb_rsqrt_fp64(double x) {
  const float s = nb_rsqrt_approx((float)x);
  if (!(s > 0.0f && s < __int_as_float(0x7f800000))) return rsqrt(x);
  const double y0 = (double)s;
  const double e = fma(-x, y0 * y0, 1.0);
  return fma(y0 * e, fma(0.375, e, 0.5), y0);
}
