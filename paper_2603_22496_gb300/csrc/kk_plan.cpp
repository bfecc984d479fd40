// kk_plan.cpp -- host side of the C ABI: validation, FP64 plan tables,
// workspace layout and the enqueue entry points.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "kk_internal.h"

namespace kk {

DeviceGuard::DeviceGuard(int dev) {
  if (cudaGetDevice(&old) != cudaSuccess) old = -1;
  if (old != dev) ok = cudaSetDevice(dev) == cudaSuccess;
}
DeviceGuard::~DeviceGuard() {
  int cur = -1;
  if (old >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != old) cudaSetDevice(old);
}

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

kk_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return KK_ERR_CUDA;
}

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kTwo32 = 4294967296.0;
constexpr double kMaxAngle = 80.0 * 3.14159265358979323846 / 180.0;
constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }


// x_ref(theta_o): the array end that makes the shear a non-negative advance.
double shear_reference(const std::vector<double> &u, double th) {
  if (th > 0) return *std::max_element(u.begin(), u.end());
  if (th < 0) return *std::min_element(u.begin(), u.end());
  return 0.0;
}

long long to_fixed32(double v) { return std::llround(v * kTwo32); }

// frac(v) as an unsigned 0.64 fixed-point fraction
unsigned long long frac64(double v) {
  double f = v - std::floor(v);
  if (f >= 1.0) f = 0.0;
  const double hi = std::floor(f * kTwo32);
  double lo = std::floor((f * kTwo32 - hi) * kTwo32);
  if (lo < 0) lo = 0;
  if (lo >= kTwo32) lo = kTwo32 - 1;
  return ((unsigned long long)hi << 32) | (unsigned long long)lo;
}

// Host staging of the plan's tables, uploaded in one allocation.
struct Blob {
  std::vector<unsigned char> bytes;
  template <typename T>
  size_t add(const std::vector<T> &v) {
    const size_t off = align_up(bytes.size());
    bytes.resize(off + std::max<size_t>(sizeof(T) * v.size(), 1));
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), sizeof(T) * v.size());
    return off;
  }
};

template <typename T>
T *at(void *base, size_t off) {
  return reinterpret_cast<T *>(static_cast<unsigned char *>(base) + off);
}

bool is_volume(const kk_plan_desc *d) {
  return d->elem_y || d->tx_angles_y || d->rx_angles_y || d->ny > 1 || d->y0 != 0.0;
}

// a plane wave (ax, ay) must propagate: sin^2 ax + sin^2 ay below sin^2(80 deg)
bool tilt_ok(double ax, double ay) {
  if (!std::isfinite(ax) || !std::isfinite(ay)) return false;
  const double sx = std::sin(ax), sy = std::sin(ay), m = std::sin(kMaxAngle);
  return sx * sx + sy * sy < m * m;
}

// unit propagation vector of a plane wave; a linear-array plan keeps
// (sin ax, 0, cos ax)
void direction(bool vol, double ax, double ay, double &sx, double &sy, double &sz) {
  if (!vol) {
    sx = std::sin(ax);
    sy = 0.0;
    sz = std::cos(ax);
    return;
  }
  sx = std::sin(ax);
  sy = std::sin(ay);
  sz = std::sqrt(1.0 - sx * sx - sy * sy);
}

// distinct values of v (ascending) and the rank of every entry among them
void distinct_ranks(const std::vector<double> &v, std::vector<double> &vals, std::vector<int> &rank) {
  vals = v;
  std::sort(vals.begin(), vals.end());
  vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
  rank.resize(v.size());
  for (size_t q = 0; q < v.size(); ++q)
    rank[q] = (int)(std::lower_bound(vals.begin(), vals.end(), v[q]) - vals.begin());
}

// Tables of the separable volumetric contraction (see k_shear_sep).
struct SepTables {
  int Lx = 0, Ly = 0, Mx = 0, My = 0;
  bool yfast = false;     // elements listed y-fastest
  bool row_major = false; // l = ls Lf + lf exactly (one bulk copy per chunk)
  std::vector<unsigned long long> phx, phy;
  std::vector<int32_t> slot, col;
};

// The element positions fill an Lx x Ly grid (each (x, y) once) and the
// receive waves in use are every combination of Mx x-tilts with My y-tilts
// (each once): then fs delta_l(o) / T = phx[ox][lx] + phy[oy][ly] with the
// per-axis shear references of Eq. (compression).  False otherwise.
bool separable_tables(const kk_plan_desc *d, int T, const std::vector<double> &u, const std::vector<double> &v,
                      const std::vector<int> &rx_used, SepTables &st) {
  const int L = (int)u.size(), Mu = (int)rx_used.size();
  std::vector<double> ux, vy, ax, ay, tx, ty;
  std::vector<int> lx, ly, ox, oy;
  distinct_ranks(u, ux, lx);
  distinct_ranks(v, vy, ly);
  st.Lx = (int)ux.size();
  st.Ly = (int)vy.size();
  if ((long long)st.Lx * st.Ly != L) return false;
  std::vector<char> seen((size_t)L, 0);
  bool xf = true, yf = true;
  for (int l = 0; l < L; ++l) {
    const int g = ly[l] * st.Lx + lx[l];
    if (seen[g]) return false;
    seen[g] = 1;
    xf = xf && g == l;
    yf = yf && lx[l] * st.Ly + ly[l] == l;
  }
  st.yfast = yf && !xf;
  st.row_major = xf || yf;
  const int Lf = st.yfast ? st.Ly : st.Lx;
  st.slot.resize(L);
  for (int l = 0; l < L; ++l) st.slot[l] = st.yfast ? lx[l] * Lf + ly[l] : ly[l] * Lf + lx[l];
  for (int a = 0; a < Mu; ++a) {
    tx.push_back(d->rx_angles[rx_used[a]]);
    ty.push_back(d->rx_angles_y ? d->rx_angles_y[rx_used[a]] : 0.0);
  }
  distinct_ranks(tx, ax, ox);
  distinct_ranks(ty, ay, oy);
  st.Mx = (int)ax.size();
  st.My = (int)ay.size();
  if ((long long)st.Mx * st.My != Mu) return false;
  st.col.assign(Mu, -1);
  for (int a = 0; a < Mu; ++a) {
    int32_t &c = st.col[st.yfast ? ox[a] * st.My + oy[a] : oy[a] * st.Mx + ox[a]];
    if (c >= 0) return false;
    c = a;
  }
  st.phx.resize((size_t)st.Mx * st.Lx);
  st.phy.resize((size_t)st.My * st.Ly);
  for (int o = 0; o < st.Mx; ++o) {
    const double sx = std::sin(ax[o]), xr = shear_reference(u, ax[o]);
    for (int l = 0; l < st.Lx; ++l)
      st.phx[(size_t)o * st.Lx + l] = frac64(d->fs * (xr - ux[l]) * sx / d->c / (double)T);
  }
  for (int o = 0; o < st.My; ++o) {
    const double sy = std::sin(ay[o]), yr = shear_reference(v, ay[o]);
    for (int l = 0; l < st.Ly; ++l)
      st.phy[(size_t)o * st.Ly + l] = frac64(d->fs * (yr - vy[l]) * sy / d->c / (double)T);
  }
  return true;
}

kk_status validate_common(const kk_plan_desc *d) {
  if (!d) { set_error("null plan description"); return KK_ERR_INVALID_ARG; }
  if (d->n_elem < 1 || !d->elem_x) { set_error("n_elem < 1 or elem_x null"); return KK_ERR_INVALID_ARG; }
  if (d->n_tx < 1 || !d->tx_angles) { set_error("n_tx < 1 or tx_angles null"); return KK_ERR_INVALID_ARG; }
  for (int i = 0; i < d->n_tx; ++i)
    if (!(std::fabs(d->tx_angles[i]) < kMaxAngle)) { set_error("transmit angle out of range (|theta| < 80 deg)"); return KK_ERR_INVALID_ARG; }
  for (int l = 0; l < d->n_elem; ++l)
    if (!std::isfinite(d->elem_x[l])) { set_error("non-finite element position"); return KK_ERR_INVALID_ARG; }
  if (!(d->c > 0) || !(d->fs > 0) || !std::isfinite(d->c) || !std::isfinite(d->fs)) { set_error("c and fs must be positive"); return KK_ERR_INVALID_ARG; }
  const kk_grid &g = d->grid;
  if (g.nx < 1 || g.nz < 1 || g.nx > 8192 || g.nz > 8192) { set_error("grid size out of range [1, 8192]"); return KK_ERR_INVALID_ARG; }
  if (!(g.dx > 0) || !(g.dz > 0) || !(g.z0 >= 0) || !std::isfinite(g.x0)) { set_error("grid needs dx > 0, dz > 0, z0 >= 0"); return KK_ERR_INVALID_ARG; }
  if (d->n_samples < 2 || d->n_samples % 2) { set_error("n_samples must be even"); return KK_ERR_INVALID_ARG; }
  if (!fft_size_supported(d->n_samples / 2)) { set_error("n_samples / 2 must be one of 128, 256, 512, 768, 1024, 1536, 2048"); return KK_ERR_UNSUPPORTED; }
  if (d->rf_dtype != KK_RF_I16 && d->rf_dtype != KK_RF_F32) { set_error("bad rf_dtype"); return KK_ERR_INVALID_ARG; }
  // the largest delay must stay well inside the 32.32 fixed-point and FP32 index range
  const double xmax = std::max(std::fabs(g.x0), std::fabs(g.x0 + g.dx * (g.nx + 64)));
  const double zmax = g.z0 + g.dz * (g.nz + 64);
  double umax = 0;
  for (int l = 0; l < d->n_elem; ++l) umax = std::max(umax, std::fabs(d->elem_x[l]));
  const double smax = d->fs / d->c * (2 * (xmax + umax) + 2 * zmax);
  if (smax > 1e6) { set_error("geometry gives delays beyond 1e6 samples"); return KK_ERR_INVALID_ARG; }
  if (is_volume(d)) {
    if (d->ny > 8192 || (long long)std::max(d->ny, 1) * g.nx * g.nz > (1ll << 31)) {
      set_error("volume size out of range (ny <= 8192, at most 2^31 voxels)");
      return KK_ERR_INVALID_ARG;
    }
    if (!std::isfinite(d->y0) || (d->ny > 1 && !(d->dy > 0 && std::isfinite(d->dy)))) {
      set_error("volume needs a finite y0 and dy > 0 when ny > 1");
      return KK_ERR_INVALID_ARG;
    }
    double vmax = 0;
    if (d->elem_y)
      for (int l = 0; l < d->n_elem; ++l) {
        if (!std::isfinite(d->elem_y[l])) { set_error("non-finite element y position"); return KK_ERR_INVALID_ARG; }
        vmax = std::max(vmax, std::fabs(d->elem_y[l]));
      }
    for (int i = 0; i < d->n_tx; ++i)
      if (!tilt_ok(d->tx_angles[i], d->tx_angles_y ? d->tx_angles_y[i] : 0.0)) {
        set_error("transmit tilts beyond sin^2 ax + sin^2 ay < sin^2(80 deg)");
        return KK_ERR_INVALID_ARG;
      }
    const double ymax = std::fabs(d->y0) + (d->ny > 1 ? d->dy * (d->ny + 64) : 0.0);
    if (d->fs / d->c * (2 * (xmax + umax) + 2 * (ymax + vmax) + 2 * zmax) > 1e6) {
      set_error("geometry gives delays beyond 1e6 samples");
      return KK_ERR_INVALID_ARG;
    }
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || d->device < 0 || d->device >= dev_count) {
    set_error("device ordinal not available");
    return KK_ERR_INVALID_ARG;
  }
  return KK_OK;
}

void fill_fft(kk_plan &p, Blob &blob, size_t &off_tw, size_t &off_rw) {
  p.fft = make_fft_plan(p.F);
  std::vector<float2> tw(std::max(p.fft.tw_count, 1));
  for (int s = 0; s < p.fft.npass; ++s) {
    const int R = p.fft.radix[s], ns = p.fft.ns[s];
    for (int k = 0; k < ns; ++k)
      for (int r = 1; r < R; ++r) {
        const long long m = ((long long)r * k) % ((long long)ns * R);
        const double a = -kTwoPi * (double)m / (double)(ns * R);
        tw[p.fft.tw_off[s] + k * (R - 1) + (r - 1)] = make_float2((float)std::cos(a), (float)std::sin(a));
      }
  }
  std::vector<float2> rw(p.F);
  for (int k = 0; k < p.F; ++k) {
    const double a = -kTwoPi * (double)k / (double)p.T;
    rw[k] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  off_tw = blob.add(tw);
  off_rw = blob.add(rw);
  std::vector<int32_t> status(1, 0);
  p.status_off = blob.add(status);
}

kk_status upload(kk_plan &p, const Blob &blob) {
  void *dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, blob.bytes.size());
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("plan table allocation failed");
    return KK_ERR_OOM;
  }
  e = cudaMemcpy(dev, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(e, "plan table upload");
  }
  p.dev_block = dev;
  return KK_OK;
}

// Pair-range split of the KK gather for a shape: the grid covers the GPU
// (~4 CTAs per SM), keeping >= 2 stages of work per slice.
int gather_split(const kk_plan &p, int rows, int stage) {
  const int tz = 4 * rows;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  const int tiles = ((p.grid.nx + kTileX - 1) / kTileX) * ((p.grid.nz + tz - 1) / tz) * p.ny;
  const int split = (4 * sms + tiles - 1) / tiles;
  const int max_by_pairs = std::max(1, (p.P / p.J) / (2 * stage));
  return std::max(1, std::min(split, max_by_pairs));
}

// Window length, tile grid and pair-range split of the KK gather for a
// (rows, stage) configuration.  The workspace reserves partial images for the
// largest split of any shape (make_kk), so it does not depend on the shape.
kk_status configure_kk_gather(kk_plan &p, int rows, int stage) {
  const kk_grid &g = p.grid;
  const int tz = 4 * rows;
  double span = 0;
  for (size_t q = 0; q < p.h_bfA.size(); ++q)
    span = std::max(span, std::fabs(p.h_bfA[q]) * (kTileX - 1) + p.h_bfB[q] * (tz - 1));
  // window: W0 = floor(min s) - 1, so a length >= span + 4 covers every read
  const int win = (int)std::ceil(span) + 4;
  if (!gather_config_supported(rows, stage, win)) {
    set_error("gather shape not available for this grid (staged window of " + std::to_string(win) +
              " samples); use fewer rows or a smaller stage");
    return KK_ERR_UNSUPPORTED;
  }
  p.bf_rows = rows;
  p.bf_stage = stage;
  p.bf_win = win;
  p.tiles_x = (g.nx + kTileX - 1) / kTileX;
  p.tiles_z = (g.nz + tz - 1) / tz;
  p.bf_split = gather_split(p, rows, stage);
  return KK_OK;
}

int choose_stage(int win) {
  // about 40 KB of staged windows per CTA, at most 32 pairs / transmits
  int st = (int)(40 * 1024 / (16 * (size_t)win));
  return std::max(1, std::min(32, st));
}

kk_status make_kk(kk_plan &p, const kk_plan_desc *d) {
  if (d->n_rx < 1 || !d->rx_angles) { set_error("n_rx < 1 or rx_angles null"); return KK_ERR_INVALID_ARG; }
  if (d->n_pairs < 1 || !d->pairs) { set_error("n_pairs < 1 or pairs null"); return KK_ERR_INVALID_ARG; }
  if (d->n_groups < 1) { set_error("n_groups < 1"); return KK_ERR_INVALID_ARG; }
  if (d->pair_weight)
    for (int q = 0; q < d->n_pairs; ++q)
      if (!std::isfinite(d->pair_weight[q])) { set_error("non-finite pair weight"); return KK_ERR_INVALID_ARG; }
  if (d->compound < KK_COMPOUND_NONE || d->compound > KK_COMPOUND_INCOHERENT) { set_error("bad compound mode"); return KK_ERR_INVALID_ARG; }
  if (d->precision < KK_PREC_F32 || d->precision > KK_PREC_F8E4M3) { set_error("bad precision"); return KK_ERR_INVALID_ARG; }
  for (int o = 0; o < d->n_rx; ++o)
    if (!(std::fabs(d->rx_angles[o]) < kMaxAngle)) { set_error("receive angle out of range (|theta| < 80 deg)"); return KK_ERR_INVALID_ARG; }
  if (p.vol)
    for (int o = 0; o < d->n_rx; ++o)
      if (!tilt_ok(d->rx_angles[o], d->rx_angles_y ? d->rx_angles_y[o] : 0.0)) {
        set_error("receive tilts beyond sin^2 ax + sin^2 ay < sin^2(80 deg)");
        return KK_ERR_INVALID_ARG;
      }
  const int P = d->n_pairs, J = d->n_groups;
  std::vector<int> gp(P, 0);
  for (int q = 0; q < P; ++q) {
    const int i = d->pairs[2 * q], o = d->pairs[2 * q + 1];
    if (i < 0 || i >= d->n_tx || o < 0 || o >= d->n_rx) { set_error("pair index out of range"); return KK_ERR_INVALID_ARG; }
    if (d->group_of_pair) {
      gp[q] = d->group_of_pair[q];
      if (gp[q] < 0 || gp[q] >= J) { set_error("group index out of range"); return KK_ERR_INVALID_ARG; }
    }
  }
  p.P = P;
  p.J = J;
  p.compound = d->compound;
  p.precision = d->precision;

  std::vector<double> u(d->elem_x, d->elem_x + p.L);
  // transmits and receive angles in use
  std::vector<int> tx_used, rx_used;
  for (int q = 0; q < P; ++q) {
    tx_used.push_back(d->pairs[2 * q]);
    rx_used.push_back(d->pairs[2 * q + 1]);
  }
  std::sort(tx_used.begin(), tx_used.end());
  tx_used.erase(std::unique(tx_used.begin(), tx_used.end()), tx_used.end());
  std::sort(rx_used.begin(), rx_used.end());
  rx_used.erase(std::unique(rx_used.begin(), rx_used.end()), rx_used.end());
  p.Nu = (int)tx_used.size();
  p.Mu = (int)rx_used.size();
  if (p.precision == KK_PREC_F16 || p.precision == KK_PREC_F8E4M3) {
    int e = 0;
    while ((1 << e) < 2 * p.T) ++e;
    p.x_scale = std::ldexp(1.0f, -e);
  }
  if (p.precision != KK_PREC_F32 && (p.L > 128 || p.Nu > 256)) {
    set_error("tensor-core precision forms need <= 128 elements and <= 256 transmits in use");
    return KK_ERR_UNSUPPORTED;
  }
  std::vector<int> tx_pos(d->n_tx, -1), rx_pos(d->n_rx, -1);
  for (int a = 0; a < p.Nu; ++a) tx_pos[tx_used[a]] = a;
  for (int a = 0; a < p.Mu; ++a) rx_pos[rx_used[a]] = a;
  p.compression = (double)p.L / (double)p.Mu;

  Blob blob;
  size_t off_tw, off_rw;
  fill_fft(p, blob, off_tw, off_rw);
  std::vector<int32_t> txu(tx_used.begin(), tx_used.end());
  const size_t off_txu = blob.add(txu);

  // shear phases: frac(fs delta_l(theta_o) / T), delta = (x_ref - u_l) sin(theta_o) / c
  std::vector<unsigned long long> phase((size_t)p.Mu * p.L);
  std::vector<double> v(p.L, 0.0);
  if (d->elem_y) v.assign(d->elem_y, d->elem_y + p.L);
  auto rx_y = [&](int o) { return d->rx_angles_y ? d->rx_angles_y[o] : 0.0; };
  auto tx_y = [&](int i) { return d->tx_angles_y ? d->tx_angles_y[i] : 0.0; };
  for (int a = 0; a < p.Mu; ++a) {
    const double th = d->rx_angles[rx_used[a]];
    const double xr = shear_reference(u, th);
    if (!p.vol) {
      for (int l = 0; l < p.L; ++l) {
        const double D = d->fs * (xr - u[l]) * std::sin(th) / d->c;  // samples
        phase[(size_t)a * p.L + l] = frac64(D / (double)p.T);
      }
      continue;
    }
    double sx, sy, sz;
    direction(true, th, rx_y(rx_used[a]), sx, sy, sz);
    const double yr = shear_reference(v, sy);
    for (int l = 0; l < p.L; ++l) {
      const double D = d->fs * ((xr - u[l]) * sx + (yr - v[l]) * sy) / d->c;  // samples
      phase[(size_t)a * p.L + l] = frac64(D / (double)p.T);
    }
  }
  const size_t off_phase = blob.add(phase);
  // separable FP32 contraction when it takes at most half the products of
  // the full one; a chunk of transmits (up to 8, at most 256 lanes along the
  // fast axis, two buffers within 110 KB of shared memory) per item
  SepTables sep;
  size_t off_w = 0, off_slot = 0, off_col = 0;
  if (p.vol && p.precision == KK_PREC_F32 && separable_tables(d, p.T, u, v, rx_used, sep)) {
    const int Lf = sep.yfast ? sep.Ly : sep.Lx, Ls = sep.yfast ? sep.Lx : sep.Ly;
    const int Mf = sep.yfast ? sep.My : sep.Mx, Ms = sep.yfast ? sep.Mx : sep.My;
    const bool bulk = sep.row_major && p.L % 2 == 0;
    const bool pays = 2LL * ((long long)Ms * Ls + (long long)Mf * Ms) * Lf <= (long long)p.L * p.Mu &&
                      Ms <= kSepMaxSlowWaves;
    int tpc = 0;
    for (int t = 1; pays && t <= 8; t *= 2)
      if (t * Lf <= 256) {
        int parts = 0, osn = 0;
        sep_split(Lf, Ms, t, parts, osn);
        if (sep_shear_smem_bytes(p.L, Lf, Ls, Mf, Ms, parts * osn, t, bulk) <= 110 * 1024) tpc = t;
      }
    if (tpc > 0) {
      p.sep_tpc = tpc;
      p.sep_Lx = sep.Lx;
      p.sep_Ly = sep.Ly;
      p.sep_Mx = sep.Mx;
      p.sep_My = sep.My;
      p.sep_yfast = sep.yfast;
      p.sep_bulk = bulk;
      // per-bin phasors exp(2 pi i frac(k phi)) in FP64, k phi mod 1 exact in
      // 0.64 fixed point, stored as FP32 pairs
      const std::vector<unsigned long long> &phf = sep.yfast ? sep.phy : sep.phx;
      const std::vector<unsigned long long> &phs = sep.yfast ? sep.phx : sep.phy;
      int parts = 0, osn = 0;
      sep_split(Lf, Ms, tpc, parts, osn);
      const int msp = parts * osn;            // Ws row: the parts' waves, zeros past Ms
      const size_t wf = (size_t)((Lf * Mf + 1) & ~1);
      const size_t per_k = wf + (size_t)Ls * msp;
      std::vector<float2> wtab((size_t)p.F * per_k, make_float2(0.f, 0.f));
      auto phasor = [](unsigned long long ph) {
        double turns = (double)ph * 0x1p-64;
        if (turns >= 0.5) turns -= 1.0;
        return make_float2((float)std::cos(2.0 * M_PI * turns), (float)std::sin(2.0 * M_PI * turns));
      };
      for (int k = 0; k < p.F; ++k) {
        float2 *w = wtab.data() + (size_t)k * per_k;
        const unsigned long long kk = (unsigned long long)k;
        for (int lf = 0; lf < Lf; ++lf)
          for (int of = 0; of < Mf; ++of) w[lf * Mf + of] = phasor(kk * phf[(size_t)of * Lf + lf]);
        for (int ls = 0; ls < Ls; ++ls)
          for (int os = 0; os < Ms; ++os) w[wf + (size_t)ls * msp + os] = phasor(kk * phs[(size_t)os * Ls + ls]);
      }
      off_w = blob.add(wtab);
      off_slot = blob.add(sep.slot);
      off_col = blob.add(sep.col);
    }
  }
  // 0.32 fixed-point copy for the reduced-precision contraction: k phi mod
  // 2^32 is then off by at most k 2^-33 turns (< 8e-7 rad for k < 1024)
  std::vector<uint32_t> phase32(phase.size());
  for (size_t q = 0; q < phase.size(); ++q) phase32[q] = (uint32_t)((phase[q] + (1ull << 31)) >> 32);
  const size_t off_phase32 = blob.add(phase32);

  std::vector<int32_t> pair_q(P);
  p.h_pair_tu.resize(P);
  p.h_pair_ou.resize(P);
  for (int q = 0; q < P; ++q) {
    p.h_pair_tu[q] = tx_pos[d->pairs[2 * q]];
    p.h_pair_ou[q] = rx_pos[d->pairs[2 * q + 1]];
    pair_q[q] = p.h_pair_tu[q] * p.Mu + p.h_pair_ou[q];
  }
  p.h_tx_used = txu;
  p.pair_q_identity = (P == p.Nu * p.Mu);
  for (int q = 0; q < P && p.pair_q_identity; ++q) p.pair_q_identity = pair_q[q] == q;
  const size_t off_pq = blob.add(pair_q);

  // gather tables, pairs stably sorted by group
  std::vector<int> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return gp[a] < gp[b]; });
  p.h_group_start.assign(J + 1, 0);
  for (int q = 0; q < P; ++q) p.h_group_start[gp[q] + 1]++;
  for (int g = 0; g < J; ++g) p.h_group_start[g + 1] += p.h_group_start[g];
  std::vector<int32_t> row(P);
  std::vector<long long> A(P), Bv(P), C(P), Yv(p.vol ? P : 0);
  std::vector<float> Af(P), Bf(P);
  const kk_grid &g = p.grid;
  const double k_s = d->fs / d->c;
  double span = 0;
  for (int s = 0; s < P; ++s) {
    const int q = order[s];
    const double ti = d->tx_angles[d->pairs[2 * q]];
    const double to = d->rx_angles[d->pairs[2 * q + 1]];
    const double xr = shear_reference(u, to);
    double a, b, c0;
    if (!p.vol) {
      const double sx = std::sin(ti) + std::sin(to);
      const double cz = std::cos(ti) + std::cos(to);
      a = k_s * g.dx * sx;
      b = k_s * g.dz * cz;
      c0 = k_s * (g.x0 * sx + g.z0 * cz - xr * std::sin(to));
    } else {
      double ix, iy, iz, ox, oy, oz;
      direction(true, ti, tx_y(d->pairs[2 * q]), ix, iy, iz);
      direction(true, to, rx_y(d->pairs[2 * q + 1]), ox, oy, oz);
      const double yr = shear_reference(v, oy);
      a = k_s * g.dx * (ix + ox);
      b = k_s * g.dz * (iz + oz);
      c0 = k_s * (g.x0 * (ix + ox) + p.y0 * (iy + oy) + g.z0 * (iz + oz) - xr * ox - yr * oy);
      Yv[s] = to_fixed32(k_s * p.dy * (iy + oy));
    }
    row[s] = q;
    p.h_bfA.push_back(a);
    p.h_bfB.push_back(b);
    A[s] = to_fixed32(a);
    Bv[s] = to_fixed32(b);
    C[s] = to_fixed32(c0);
    Af[s] = (float)a;
    Bf[s] = (float)b;
  }
  // Samples of each record the gather can stage, for record trimming.  A
  // tile's window starts at W0 = floor(min over the tile of s) - 1 (the
  // 32.32 tables, as the kernels compute it) and the staging reads y[k] and
  // y[k+1] for k in [W0, W0 + win): samples [W0, W0 + win].  W0 is monotone
  // in the tile's origin, so its extremes are at the corner tiles; every
  // launch shape (4-, 8-, 16- and 32-row tiles) is covered.
  std::vector<int2> rng(P, make_int2(0, 0));
  if (!p.vol) {
    const int tzs[3] = {8, 16, 32};
    long long wins[3];
    for (int v = 0; v < 3; ++v) {
      double sp = 0;  // as configure_kk_gather: span over every pair
      for (int q = 0; q < P; ++q) sp = std::max(sp, std::fabs(p.h_bfA[q]) * (kTileX - 1) + p.h_bfB[q] * (tzs[v] - 1));
      wins[v] = (long long)std::ceil(sp) + 4;
    }
    const long long x_last = (long long)((g.nx + kTileX - 1) / kTileX - 1) * kTileX;
    for (int s = 0; s < P; ++s) {
      long long lo = LLONG_MAX, hi = LLONG_MIN;
      for (int v = 0; v < 3; ++v) {
        const long long z_last = (long long)((g.nz + tzs[v] - 1) / tzs[v] - 1) * tzs[v];
        for (long long x0 : {0LL, x_last})
          for (long long z0 : {0LL, z_last}) {
            const long long smin = C[s] + Bv[s] * z0 + A[s] * (A[s] >= 0 ? x0 : x0 + kTileX - 1);
            const long long w0 = (smin >> 32) - 1;
            lo = std::min(lo, w0);
            hi = std::max(hi, w0 + wins[v] + 1);
          }
      }
      lo = std::max(0LL, std::min(lo, (long long)p.T));
      hi = std::max(lo, std::min(hi, (long long)p.T));
      rng[row[s]] = make_int2((int)lo, (int)hi);
      if (hi > lo) p.trim_bytes += 16 * (size_t)((hi + 1) / 2 - lo / 2);  // sample pairs overlapping [lo, hi)
    }
  }
  const size_t off_rng = blob.add(rng);
  const size_t off_row = blob.add(row), off_A = blob.add(A), off_B = blob.add(Bv), off_C = blob.add(C);
  const size_t off_Af = blob.add(Af), off_Bf = blob.add(Bf);
  const size_t off_Y = p.vol ? blob.add(Yv) : 0;
  size_t off_W = 0;
  if (d->pair_weight) {  // caller's pair order: rows of rf_theta
    std::vector<float> wv(P);
    for (int q = 0; q < P; ++q) wv[q] = (float)d->pair_weight[q];
    off_W = blob.add(wv);
    p.h_pair_w = wv;
  }
  std::vector<int32_t> gs(p.h_group_start.begin(), p.h_group_start.end());
  const size_t off_gs = blob.add(gs);

  // workspace: X [F][Nu][L] (complex, precision-dependent width), Y [F][Nu][Mu]
  // complex FP32, then the gather's partial images
  size_t off = 0;
  p.ws_X = off;
  off = align_up(off + (size_t)spectrum_bytes(p.precision) * p.F * p.Nu * p.L);
  p.ws_Y = off;
  off = align_up(off + sizeof(float2) * (size_t)p.F * p.Nu * p.Mu);
  p.ws_part = off;
  (void)span;
  // default launch shape: 32 x 16 tiles, 16 pairs per stage (8 when the
  // window is long); coarse grids fall back to smaller stages
  kk_status cst = KK_ERR_UNSUPPORTED;
  for (const int *rs : {(const int[2]){4, 16}, (const int[2]){4, 8}, (const int[2]){4, 4},
                        (const int[2]){2, 8}, (const int[2]){2, 4}})
    if ((cst = configure_kk_gather(p, rs[0], rs[1])) == KK_OK) break;
  if (cst != KK_OK) return cst;
  // partial images for the largest split any shape can take
  int max_split = 1;
  for (int rows : {2, 4, 8})
    for (int stage : {4, 8, 16}) max_split = std::max(max_split, gather_split(p, rows, stage));
  p.ws_total = max_split > 1 ? align_up(off + sizeof(float2) * (size_t)max_split * p.J * p.grid.nx * p.grid.nz *
                                             (size_t)p.ny)
                             : off;

  kk_status st = upload(p, blob);
  if (st != KK_OK) return st;
  void *b = p.dev_block;
  p.t.fft_tw = at<float2>(b, off_tw);
  p.t.rfft_w = at<float2>(b, off_rw);
  p.t.tx_used = at<int32_t>(b, off_txu);
  p.t.phase = at<unsigned long long>(b, off_phase);
  p.t.phase32 = at<uint32_t>(b, off_phase32);
  if (p.sep_Lx > 0) {
    p.t.sep_w = at<float2>(b, off_w);
    p.t.sep_slot = at<int32_t>(b, off_slot);
    p.t.sep_col = at<int32_t>(b, off_col);
  }
  p.t.pair_q = at<int32_t>(b, off_pq);
  p.t.bf_row = at<int32_t>(b, off_row);
  p.t.bf_A = at<long long>(b, off_A);
  p.t.bf_B = at<long long>(b, off_B);
  p.t.bf_C = at<long long>(b, off_C);
  p.t.bf_Y = p.vol ? at<long long>(b, off_Y) : nullptr;
  p.t.bf_Af = at<float>(b, off_Af);
  p.t.bf_Bf = at<float>(b, off_Bf);
  p.t.pair_w = d->pair_weight ? at<float>(b, off_W) : nullptr;
  p.t.group_start = at<int32_t>(b, off_gs);
  p.t.rec_range = at<int2>(b, off_rng);
  p.t.status = at<int>(b, p.status_off);
  return KK_OK;
}

kk_status make_das(kk_plan &p, const kk_plan_desc *d) {
  if (!std::isfinite(d->f_number) || (d->aperture != KK_APERTURE_BOXCAR && d->aperture != KK_APERTURE_HANN)) {
    set_error("bad receive aperture (finite f_number, KK_APERTURE_BOXCAR or KK_APERTURE_HANN)");
    return KK_ERR_INVALID_ARG;
  }
  if (p.vol && d->f_number > 0) {
    set_error("volumetric DAS sums the full aperture (f_number 0)");
    return KK_ERR_UNSUPPORTED;
  }
  p.das_two_f = d->f_number > 0 ? (float)(2.0 * d->f_number) : 0.f;
  p.das_window = d->aperture;
  p.is_das = true;
  p.J = 1;
  p.P = p.N * p.L;
  p.Nu = p.N;
  p.Mu = 0;
  p.compound = KK_COMPOUND_NONE;
  p.precision = KK_PREC_F32;
  p.compression = 1.0;
  Blob blob;
  size_t off_tw, off_rw;
  fill_fft(p, blob, off_tw, off_rw);
  std::vector<int32_t> txu(p.N);
  std::iota(txu.begin(), txu.end(), 0);
  const size_t off_txu = blob.add(txu);
  const kk_grid &g = p.grid;
  const double k_s = d->fs / d->c;
  std::vector<long long> A(p.N), Bv(p.N), C(p.N), Yv(p.vol ? p.N : 0);
  std::vector<float> Af(p.N), Bf(p.N);
  // staged kernel: 32 x 16 tiles, window from the transmit-delay span plus the
  // receive-delay span, which the tile diameter bounds (|grad R| <= 1, also
  // within one y slice of a volume); windows over 256 entries go to the
  // synchronous 32 x 32 kernel (linear arrays only)
  const double diam16 = std::hypot(g.dx * (kTileX - 1), g.dz * 15.0);
  double span_in16 = 0, span_in32 = 0;
  for (int i = 0; i < p.N; ++i) {
    double sx, sy, sz;
    direction(p.vol, d->tx_angles[i], d->tx_angles_y ? d->tx_angles_y[i] : 0.0, sx, sy, sz);
    const double a = k_s * g.dx * sx, b = k_s * g.dz * sz;
    const double c0 = k_s * (g.x0 * sx + p.y0 * sy + g.z0 * sz);
    if (p.vol) Yv[i] = to_fixed32(k_s * p.dy * sy);
    A[i] = to_fixed32(a);
    Bv[i] = to_fixed32(b);
    C[i] = to_fixed32(c0);
    Af[i] = (float)a;
    Bf[i] = (float)b;
    span_in16 = std::max(span_in16, std::fabs(a) * (kTileX - 1) + b * 15.0);
    span_in32 = std::max(span_in32, std::fabs(a) * (kTileX - 1) + b * (kTileZ - 1));
  }
  const int win16 = (int)std::ceil(span_in16 + k_s * diam16) + 6;
  const int stage16 = das_staged_stage(win16);
  if (p.vol && stage16 == 0) {
    set_error("volumetric DAS needs staged windows of at most 256 samples (a finer x / z pitch)");
    return KK_ERR_UNSUPPORTED;
  }
  const int TZ = stage16 > 0 ? 16 : kTileZ;
  p.tiles_x = (g.nx + kTileX - 1) / kTileX;
  p.tiles_z = (g.nz + TZ - 1) / TZ;
  auto split_df = [](double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
  };
  std::vector<float2> xs(p.tiles_x * kTileX), zs(p.tiles_z * TZ), us(p.L);
  for (size_t k = 0; k < xs.size(); ++k) xs[k] = split_df(k_s * (g.x0 + g.dx * (double)k));
  for (size_t k = 0; k < zs.size(); ++k) zs[k] = split_df(k_s * (g.z0 + g.dz * (double)k));
  for (int l = 0; l < p.L; ++l) us[l] = split_df(k_s * d->elem_x[l]);
  std::vector<float2> ysl(p.vol ? p.ny : 0), usy(p.vol ? p.L : 0);
  for (int k = 0; k < (int)ysl.size(); ++k) ysl[k] = split_df(k_s * (p.y0 + p.dy * (double)k));
  for (int l = 0; l < (int)usy.size(); ++l) usy[l] = split_df(k_s * (d->elem_y ? d->elem_y[l] : 0.0));
  const size_t off_A = blob.add(A), off_B = blob.add(Bv), off_C = blob.add(C);
  const size_t off_Af = blob.add(Af), off_Bf = blob.add(Bf);
  const size_t off_xs = blob.add(xs), off_zs = blob.add(zs), off_us = blob.add(us);
  const size_t off_Y = p.vol ? blob.add(Yv) : 0, off_ys = p.vol ? blob.add(ysl) : 0;
  const size_t off_usy = p.vol ? blob.add(usy) : 0;
  if (stage16 > 0) {
    p.bf_rows = 4;
    p.bf_win = win16;
    p.bf_stage = stage16;
  } else {
    const double span_out = k_s * (g.dx * (kTileX - 1) + g.dz * (kTileZ - 1));
    p.bf_rows = 8;
    p.bf_win = (int)std::ceil(span_in32 + span_out) + 6;
    p.bf_stage = choose_stage(p.bf_win);
  }
  // split the element loop so the grid covers the GPU (~4 CTAs per SM)
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  const int tiles = p.tiles_x * p.tiles_z * p.ny;
  p.bf_split = std::max(1, std::min((4 * sms + tiles - 1) / tiles, p.L / 4));
  // workspace: X [F][N*L], analytic channels y [N*L][T], partial images
  size_t off = 0;
  p.ws_X = off;
  off = align_up(off + sizeof(float2) * (size_t)p.F * p.N * p.L);
  p.ws_Y = off;
  off = align_up(off + sizeof(float2) * (size_t)p.N * p.L * p.T);
  p.ws_part = off;
  if (p.bf_split > 1) off = align_up(off + sizeof(float2) * (size_t)p.bf_split * g.nx * g.nz * p.ny);
  p.ws_total = off;
  kk_status st = upload(p, blob);
  if (st != KK_OK) return st;
  void *b = p.dev_block;
  p.t.fft_tw = at<float2>(b, off_tw);
  p.t.rfft_w = at<float2>(b, off_rw);
  p.t.tx_used = at<int32_t>(b, off_txu);
  p.t.das_A = at<long long>(b, off_A);
  p.t.das_B = at<long long>(b, off_B);
  p.t.das_C = at<long long>(b, off_C);
  p.t.das_Af = at<float>(b, off_Af);
  p.t.das_Bf = at<float>(b, off_Bf);
  p.t.xs = at<float2>(b, off_xs);
  p.t.zs = at<float2>(b, off_zs);
  p.t.us = at<float2>(b, off_us);
  if (p.vol) {
    p.t.das_Y = at<long long>(b, off_Y);
    p.t.ys = at<float2>(b, off_ys);
    p.t.us_y = at<float2>(b, off_usy);
  }
  p.t.status = at<int>(b, p.status_off);
  return KK_OK;
}

kk_status create(kk_plan **out, const kk_plan_desc *d, bool das) {
  if (!out) { set_error("null output pointer"); return KK_ERR_INVALID_ARG; }
  *out = nullptr;
  kk_status st = validate_common(d);
  if (st != KK_OK) return st;
  DeviceGuard guard(d->device);
  if (!guard.ok) { set_error("cudaSetDevice failed"); return KK_ERR_CUDA; }
  kk_plan *p = new (std::nothrow) kk_plan();
  if (!p) { set_error("host allocation failed"); return KK_ERR_OOM; }
  p->device = d->device;
  p->L = d->n_elem;
  p->N = d->n_tx;
  p->T = d->n_samples;
  p->F = d->n_samples / 2;
  p->grid = d->grid;
  p->c = d->c;
  p->fs = d->fs;
  p->rf_dtype = d->rf_dtype;
  p->vol = is_volume(d);
  p->ny = std::max(d->ny, 1);
  p->y0 = d->y0;
  p->dy = d->ny > 1 ? d->dy : 0.0;
  try {
    st = das ? make_das(*p, d) : make_kk(*p, d);
  } catch (const std::bad_alloc &) {
    set_error("host allocation failed");
    st = KK_ERR_OOM;
  } catch (...) {
    set_error("unexpected host exception in plan creation");
    st = KK_ERR_INVALID_ARG;
  }
  if (st != KK_OK) {
    if (p->dev_block) cudaFree(p->dev_block);
    delete p;
    return st;
  }
  *out = p;
  return KK_OK;
}

kk_status check_plan(const kk_plan *p, bool want_das) {
  if (!p) { set_error("null plan"); return KK_ERR_INVALID_ARG; }
  if (p->is_das != want_das) { set_error(want_das ? "expected a DAS plan" : "expected a KK plan"); return KK_ERR_INVALID_ARG; }
  return KK_OK;
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

}  // namespace

kk_status enqueue_decompose(const kk_plan *p, const void *rf, void *rf_theta, void *ws, cudaStream_t s,
                            bool side_by_side) {
  NvtxRange range("kk_decompose");
  void *X = at<unsigned char>(ws, p->ws_X);
  float2 *Y = at<float2>(ws, p->ws_Y);
  cudaError_t e;
  {
    NvtxRange r("kk_decompose/spectrum");
    e = launch_spectrum(*p, rf, X, p->Nu, p->t.tx_used, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "spectrum launch");
  {
    NvtxRange r("kk_decompose/contraction");
    e = launch_shear(*p, X, Y, s, side_by_side);
  }
  if (e != cudaSuccess) return cuda_fail(e, "shear launch");
  NvtxRange r("kk_decompose/inverse");
  e = launch_inverse(*p, Y, p->Nu * p->Mu, p->pair_q_identity ? nullptr : p->t.pair_q, p->P, (float2 *)rf_theta, s,
                     p->t.pair_w);
  if (e != cudaSuccess) return cuda_fail(e, "inverse launch");
  return KK_OK;
}

cudaError_t launch_shear(const kk_plan &p, const void *X, float2 *Y, cudaStream_t s, bool side_by_side) {
  return (p.precision == KK_PREC_F32) ? launch_shear_f32(p, (const float2 *)X, Y, s, side_by_side)
                                      : launch_shear_tc(p, X, Y, s);
}

kk_status check_beamform_args(const kk_plan *p, const void *rf_theta, const void *B, const float *I) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (!rf_theta || !B) { set_error("null buffer"); return KK_ERR_INVALID_ARG; }
  if (p->compound != KK_COMPOUND_NONE && !I) { set_error("compound mode set but I is null"); return KK_ERR_INVALID_ARG; }
  if (!aligned(rf_theta, 16)) { set_error("rf_theta must be 16-byte aligned"); return KK_ERR_INVALID_ARG; }
  return KK_OK;
}

kk_status enqueue_beamform(const kk_plan *p, const void *rf_theta, void *B, float *I, void *ws, cudaStream_t s) {
  NvtxRange range("kk_beamform");
  float2 *part = (p->bf_split > 1) ? at<float2>(ws, p->ws_part) : nullptr;
  cudaError_t e = launch_kk_gather(*p, (const float2 *)rf_theta, (float2 *)B, I, part, s);
  if (e != cudaSuccess) return cuda_fail(e, "kk gather launch");
  return KK_OK;
}

namespace {

kk_status enqueue_das(const kk_plan *p, const void *rf, void *B, float *I, void *ws, cudaStream_t s) {
  NvtxRange range("das_beamform");
  float2 *X = at<float2>(ws, p->ws_X);
  float2 *y = at<float2>(ws, p->ws_Y);
  cudaError_t e;
  {
    NvtxRange r("das_beamform/analytic");
    e = launch_spectrum(*p, rf, X, p->N, p->t.tx_used, s);
    if (e == cudaSuccess) e = launch_inverse(*p, X, p->N * p->L, nullptr, p->N * p->L, y, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "analytic signal launch");
  float2 *part = (p->bf_split > 1) ? at<float2>(ws, p->ws_part) : nullptr;
  NvtxRange r("das_beamform/gather");
  e = launch_das_gather(*p, y, (float2 *)B, I, part, s);
  if (e != cudaSuccess) return cuda_fail(e, "das gather launch");
  return KK_OK;
}

}  // namespace
}  // namespace kk

using namespace kk;

extern "C" {

const char *kk_last_error(void) { return g_err.c_str(); }

const char *kk_version(void) { return "kkbeam 0.1 (sm_103a)"; }

kk_status kk_plan_create(kk_plan **out, const kk_plan_desc *d) { return create(out, d, false); }

kk_status das_plan_create(kk_plan **out, const kk_plan_desc *d) { return create(out, d, true); }

void kk_plan_destroy(kk_plan *p) {
  if (!p) return;
  if (p->dev_block) {
    DeviceGuard guard(p->device);
    cudaFree(p->dev_block);
  }
  delete p;
}

kk_status kk_plan_set_gather(kk_plan *p, int32_t rows, int32_t stage) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (!((rows == 2 || rows == 4 || rows == 8) && (stage == 4 || stage == 8 || stage == 16))) {
    set_error("gather configuration must be rows in {2, 4, 8}, stage in {4, 8, 16}");
    return KK_ERR_INVALID_ARG;
  }
  const int r0 = p->bf_rows, s0 = p->bf_stage;
  st = configure_kk_gather(*p, rows, stage);
  if (st != KK_OK) configure_kk_gather(*p, r0, s0);
  return st;
}

kk_status kk_plan_set_trim(kk_plan *p, int32_t on) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (on != 0 && on != 1) { set_error("trim must be 0 or 1"); return KK_ERR_INVALID_ARG; }
  if (on && p->vol) {
    set_error("record trimming is for linear-array plans (volumetric plans keep full records)");
    return KK_ERR_UNSUPPORTED;
  }
  p->trim = on != 0;
  return KK_OK;
}

kk_status kk_plan_status(const kk_plan *p, int32_t *status) {
  if (!p || !status) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  int32_t v = 0, zero = 0;
  cudaError_t e = cudaMemcpy(&v, p->t.status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  e = cudaMemcpy(p->t.status, &zero, sizeof(zero), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "status reset");
  *status = v;
  return KK_OK;
}

kk_status kk_plan_workspace_size(const kk_plan *p, size_t *bytes) {
  if (!p || !bytes) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  *bytes = p->ws_total;
  return KK_OK;
}

kk_status kk_plan_get_info(const kk_plan *p, kk_plan_info *info) {
  if (!p || !info) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  std::memset(info, 0, sizeof(*info));
  info->n_elem = p->L;
  info->n_tx = p->N;
  info->n_samples = p->T;
  info->n_bins = p->F;
  info->n_tx_used = p->Nu;
  info->n_rx_used = p->Mu;
  info->n_pairs = p->P;
  info->n_groups = p->J;
  info->nx = p->grid.nx;
  info->nz = p->grid.nz;
  info->is_das = p->is_das ? 1 : 0;
  info->workspace_bytes = p->ws_total;
  info->rf_bytes = (size_t)p->N * p->L * p->T * (p->rf_dtype == KK_RF_I16 ? 2 : 4);
  info->rf_theta_bytes = p->is_das ? 0 : (size_t)p->P * p->T * 8;
  info->image_bytes = (size_t)p->J * p->grid.nx * p->grid.nz * p->ny * 8;
  info->intensity_bytes = (size_t)p->grid.nx * p->grid.nz * p->ny * 4;
  info->ny = p->ny;
  info->is_volume = p->vol ? 1 : 0;
  info->sep_lx = p->sep_Lx;
  info->sep_ly = p->sep_Ly;
  info->sep_mx = p->sep_Mx;
  info->sep_my = p->sep_My;
  info->compression_factor = p->compression;
  info->launches_decompose = p->is_das ? 0 : 3;
  info->launches_beamform = (p->is_das ? 2 : 0) + (p->bf_split > 1 ? 2 : 1);
  info->gather_rows = p->bf_rows;
  info->gather_stage = p->bf_stage;
  info->gather_split = p->bf_split;
  info->records_trimmed = p->trim ? 1 : 0;
  info->rf_theta_stored_bytes = p->is_das ? 0 : (p->trim ? p->trim_bytes : (size_t)p->P * p->T * 8);
  return KK_OK;
}

kk_status kk_decompose(const kk_plan *p, const void *d_rf, void *d_rf_theta, void *d_ws, void *stream) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (!d_rf || !d_rf_theta || !d_ws) { set_error("null buffer"); return KK_ERR_INVALID_ARG; }
  if (!aligned(d_rf, 16) || !aligned(d_rf_theta, 16) || !aligned(d_ws, kAlign)) { set_error("buffers must be 16-byte aligned (workspace 256)"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  return enqueue_decompose(p, d_rf, d_rf_theta, d_ws, (cudaStream_t)stream);
}

kk_status kk_spectrum(const kk_plan *p, const void *d_rf, void *d_X, void *stream) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (!d_rf || !d_X) { set_error("null buffer"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  cudaError_t e = launch_spectrum(*p, d_rf, d_X, p->Nu, p->t.tx_used, (cudaStream_t)stream);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "spectrum launch");
}

kk_status kk_shear(const kk_plan *p, const void *d_X, void *d_Y, void *stream) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (!d_X || !d_Y) { set_error("null buffer"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  cudaError_t e = (p->precision == KK_PREC_F32)
                      ? launch_shear_f32(*p, (const float2 *)d_X, (float2 *)d_Y, (cudaStream_t)stream)
                      : launch_shear_tc(*p, d_X, (float2 *)d_Y, (cudaStream_t)stream);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "shear launch");
}

kk_status kk_inverse(const kk_plan *p, const void *d_Y, void *d_rf_theta, void *stream) {
  kk_status st = check_plan(p, false);
  if (st != KK_OK) return st;
  if (!d_Y || !d_rf_theta) { set_error("null buffer"); return KK_ERR_INVALID_ARG; }
  if (!aligned(d_rf_theta, 16)) { set_error("rf_theta must be 16-byte aligned"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  cudaError_t e = launch_inverse(*p, (const float2 *)d_Y, p->Nu * p->Mu, p->pair_q_identity ? nullptr : p->t.pair_q, p->P,
                                 (float2 *)d_rf_theta, (cudaStream_t)stream, p->t.pair_w);
  return e == cudaSuccess ? KK_OK : cuda_fail(e, "inverse launch");
}

kk_status kk_beamform(const kk_plan *p, const void *d_rf_theta, void *d_B, float *d_I, void *d_ws, void *stream) {
  kk_status st = check_beamform_args(p, d_rf_theta, d_B, d_I);
  if (st != KK_OK) return st;
  if (p->bf_split > 1 && !d_ws) { set_error("workspace required"); return KK_ERR_INVALID_ARG; }
  if (d_ws && !aligned(d_ws, kAlign)) { set_error("workspace must be 256-byte aligned"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  return enqueue_beamform(p, d_rf_theta, d_B, d_I, d_ws, (cudaStream_t)stream);
}

kk_status das_beamform(const kk_plan *p, const void *d_rf, void *d_B, float *d_I, void *d_ws, void *stream) {
  kk_status st = check_plan(p, true);
  if (st != KK_OK) return st;
  if (!d_rf || !d_B || !d_ws) { set_error("null buffer"); return KK_ERR_INVALID_ARG; }
  if (!aligned(d_rf, 16) || !aligned(d_ws, kAlign)) { set_error("buffers must be 16-byte aligned (workspace 256)"); return KK_ERR_INVALID_ARG; }
  DeviceGuard guard(p->device);
  return enqueue_das(p, d_rf, d_B, d_I, d_ws, (cudaStream_t)stream);
}

kk_status kk_run_host_scratch_size(const kk_plan *p, size_t *bytes) {
  if (!p || !bytes) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  kk_plan_info info;
  kk_plan_get_info(p, &info);
  size_t off = align_up(info.rf_bytes);
  off += align_up(info.rf_theta_bytes);
  off += align_up(info.image_bytes);
  off += align_up(info.intensity_bytes);
  off += align_up(p->ws_total);
  *bytes = off;
  return KK_OK;
}

kk_status kk_run_host(const kk_plan *p, const void *h_rf, void *h_B, float *h_I, void *d_scratch, void *stream) {
  if (!p || !h_rf || !h_B || !d_scratch) { set_error("null argument"); return KK_ERR_INVALID_ARG; }
  if (!aligned(d_scratch, kAlign)) { set_error("scratch must be 256-byte aligned"); return KK_ERR_INVALID_ARG; }
  kk_plan_info info;
  kk_plan_get_info(p, &info);
  unsigned char *base = (unsigned char *)d_scratch;
  size_t off = 0;
  void *d_rf = base + off; off += align_up(info.rf_bytes);
  void *d_rt = base + off; off += align_up(info.rf_theta_bytes);
  void *d_B = base + off; off += align_up(info.image_bytes);
  float *d_I = (float *)(base + off); off += align_up(info.intensity_bytes);
  void *d_ws = base + off;
  DeviceGuard guard(p->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(d_rf, h_rf, info.rf_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "rf upload");
  const bool want_I = p->is_das || p->compound != KK_COMPOUND_NONE;
  kk_status st;
  if (p->is_das) {
    st = enqueue_das(p, d_rf, d_B, want_I ? d_I : nullptr, d_ws, s);
  } else {
    st = enqueue_decompose(p, d_rf, d_rt, d_ws, s);
    if (st == KK_OK) st = enqueue_beamform(p, d_rt, d_B, want_I ? d_I : nullptr, d_ws, s);
  }
  if (st != KK_OK) return st;
  e = cudaMemcpyAsync(h_B, d_B, info.image_bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "image download");
  if (h_I && want_I) {
    e = cudaMemcpyAsync(h_I, d_I, info.intensity_bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "intensity download");
  }
  return KK_OK;
}

kk_status kk_scheme_angles(int32_t kind, int32_t n_tx, const double *tx, double dtheta, int32_t M,
                           double j, double *out_rx) {
  if (!out_rx || M < 1) { set_error("M < 1 or null output"); return KK_ERR_INVALID_ARG; }
  if (kind == KK_SCHEME_SAME) {
    if (!tx || M != n_tx) { set_error("SAME scheme needs tx and M == n_tx"); return KK_ERR_INVALID_ARG; }
    for (int m = 0; m < M; ++m) out_rx[m] = tx[m];
    return KK_OK;
  }
  if (!(dtheta > 0) || !std::isfinite(dtheta)) { set_error("dtheta must be positive"); return KK_ERR_INVALID_ARG; }
  const int half = n_tx / 2;
  if (kind == KK_SCHEME_CONFOCAL && half < 1) { set_error("confocal scheme needs floor(n_tx/2) >= 1"); return KK_ERR_INVALID_ARG; }
  if (kind != KK_SCHEME_VERNIER && kind != KK_SCHEME_SHIFTED && kind != KK_SCHEME_CONFOCAL) {
    set_error("unknown scheme");
    return KK_ERR_INVALID_ARG;
  }
  for (int m = 0; m < M; ++m) {
    const double o = (double)m - 0.5 * (double)(M - 1);   // receive index, Section II-C
    const double ao = std::fabs(o);
    const double sg = (o > 0) ? 1.0 : (o < 0 ? -1.0 : 0.0);
    double shift = 0.0;
    if (kind == KK_SCHEME_SHIFTED) shift = j;                           // Eq. (uniform)
    if (kind == KK_SCHEME_CONFOCAL) shift = std::fmod(std::floor(ao), (double)half);  // Eq. (confocal)
    out_rx[m] = sg * dtheta * (2.0 * ao / (double)M + shift);
  }
  return KK_OK;
}

}  // extern "C"
