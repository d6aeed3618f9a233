// Domain decomposition of one grid into bricks with a halo exchange per RK
// stage (declared in include/mhd.h, "domain decomposition").
//
// The paper splits its domain between processes and, at every stage, packs
// the boundary data each neighbour needs into device buffers, exchanges them
// with non-blocking sends and receives -- 8 neighbours in 2D, 26 in 3D,
// diagonal ones included -- and unpacks them into the ghost zones (§3.4
// "Multi GPU communication", Fig. par_ex).  Here every brick is a full
// single-grid context (mhd_ctx) whose ghost fill is replaced by that
// exchange:
//
//   pack     one kernel per brick gathers, for each neighbour, the box of its
//            interior that the neighbour's ghost shell needs into the brick's
//            send buffer;
//   exchange one device copy per (brick, neighbour) pair from the sender's
//            send buffer into the receiver's receive buffer -- the transfer
//            that a peer copy or a message carries between GPUs;
//   unpack   one kernel per brick scatters its receive buffer into its ghost
//            shell; then the brick's sides on an outflow boundary of the
//            whole grid get the outflow fill.
//
// Every ghost slot of a brick then holds what the undivided grid holds at
// the same global position, so each brick executes exactly the undivided
// grid's arithmetic on its cells, and the CFL step -- the least of the
// bricks' steps, cfl / max rate being monotone in the rate -- is the
// undivided grid's to the bit.  All bricks share one device and one stream;
// a step is captured once in a CUDA graph and replayed.
#include <algorithm>
#include <climits>
#include <cmath>
#include <new>
#include <vector>

#include "mhd.h"
#include "mhd_ctx.cuh"
#include "mhd_host.cuh"
#include "mhd_kernels.cuh"

using namespace mhd;

namespace {

constexpr int kMaxBoxes = 26;

// ---------------------------------------------------------------------------
// Partition and halo boxes (host only; no device work)
// ---------------------------------------------------------------------------
struct Part {
  int ndim, G;
  int N[3];      // cells of the whole grid per axis (1 on inactive axes)
  int p[3];      // bricks per axis
  int per[3];    // periodic axis
};

int make_part(const mhd_config* cfg, const int parts[3], Part& P) {
  int rc = validate(cfg);
  if (rc) return rc;
  if (!parts || cfg->divb != MHD_DIVB_CT) return MHD_ERR_ARG;
  P.ndim = cfg->ndim;
  P.G = cfg->recon == MHD_RECON_PLM ? 2 : 3;
  const int N[3] = {cfg->nx, cfg->ny, cfg->ndim == 3 ? cfg->nz : 1};
  for (int d = 0; d < 3; d++) {
    P.N[d] = N[d];
    P.p[d] = parts[d];
    P.per[d] = d < cfg->ndim ? cfg->bc[2 * d] == MHD_BC_PERIODIC : 1;
    if (parts[d] < 1 || (d >= cfg->ndim && parts[d] != 1)) return MHD_ERR_ARG;
    // every brick needs at least G + 1 cells: its first G + 1 and last G
    // cells are what its neighbours' ghost shells copy
    if (d < cfg->ndim && N[d] / parts[d] < P.G + 1) return MHD_ERR_ARG;
  }
  if ((long long)P.p[0] * P.p[1] * P.p[2] > 4096) return MHD_ERR_ARG;
  return MHD_OK;
}

int nbricks(const Part& P) { return P.p[0] * P.p[1] * P.p[2]; }

void brick_coord(const Part& P, int b, int c[3]) {
  c[0] = b % P.p[0];
  c[1] = (b / P.p[0]) % P.p[1];
  c[2] = b / (P.p[0] * P.p[1]);
}

// Axis d split into p near-equal parts: the first N % p parts get one more cell.
void brick_span(const Part& P, int d, int c, int& lo, int& n) {
  const int base = P.N[d] / P.p[d], rem = P.N[d] % P.p[d];
  n = base + (c < rem ? 1 : 0);
  lo = c * base + std::min(c, rem);
}

void brick_box(const Part& P, int b, int lo[3], int n[3]) {
  int c[3];
  brick_coord(P, b, c);
  for (int d = 0; d < 3; d++) brick_span(P, d, c[d], lo[d], n[d]);
}

// The brick next to brick b in direction o (-1, 0, +1 per axis), wrapping
// periodic axes; -1 across an outflow boundary of the whole grid.
int neighbour(const Part& P, int b, const int o[3]) {
  int c[3];
  brick_coord(P, b, c);
  for (int d = 0; d < 3; d++) {
    c[d] += o[d];
    if (c[d] < 0 || c[d] >= P.p[d]) {
      if (!P.per[d]) return -1;
      c[d] = (c[d] + P.p[d]) % P.p[d];
    }
  }
  return c[0] + P.p[0] * (c[1] + P.p[1] * c[2]);
}

// Neighbour directions in a fixed order (x fastest), all-zero excluded.
int directions(const Part& P, int dirs[kMaxBoxes][3]) {
  int m = 0;
  for (int oz = -1; oz <= 1; oz++)
    for (int oy = -1; oy <= 1; oy++)
      for (int ox = -1; ox <= 1; ox++) {
        if (ox == 0 && oy == 0 && oz == 0) continue;
        if (P.ndim == 2 && oz != 0) continue;
        dirs[m][0] = ox;
        dirs[m][1] = oy;
        dirs[m][2] = oz;
        m++;
      }
  return m;
}

// Boxes of brick b in its own padded coordinates (cell index -G..n+G), in
// direction order, with their offsets in slots:
//   send: the part of b's interior that the neighbour in direction o needs:
//         per axis, o = +1: [n-G, n-1];  o = -1: [0, G];  o = 0: [0, n-1];
//   recv: b's ghost region in direction o, filled by that neighbour:
//         per axis, o = -1: [-G, -1];    o = +1: [n, n+G]; o = 0: [0, n-1].
// The box b sends in direction o has the extents of the box its neighbour
// receives in direction -o (the slot n+G of the upper ghost layers is the last
// face of a face array, so that side has G + 1 slots).  On an outflow axis the
// last brick's slot n holds the upper boundary face of that axis's face array
// (evolved like any face): its o = 0 boxes along that axis are [0, n], so a
// transverse neighbour's ghost columns get that face too; the cells and the
// other fields of the slot are ghosts that the receiver's own outflow fill
// then sets.
int halo_boxes(const Part& P, int b, bool send, mhd_halo_box* out, int max, int* count, long long* slots) {
  int lo[3], n[3], cb[3];
  brick_box(P, b, lo, n);
  brick_coord(P, b, cb);
  int dirs[kMaxBoxes][3];
  const int nd = directions(P, dirs);
  int m = 0;
  long long off = 0;
  for (int r = 0; r < nd; r++) {
    const int* o = dirs[r];
    const int peer = neighbour(P, b, o);
    if (peer < 0) continue;
    if (m >= max) return MHD_ERR_ARG;
    mhd_halo_box& x = out[m++];
    x.peer = peer;
    for (int d = 0; d < 3; d++) {
      x.dir[d] = o[d];
      if (d >= P.ndim) {
        x.lo[d] = 0;
        x.ext[d] = 1;
      } else if (o[d] == 0) {
        x.lo[d] = 0;
        x.ext[d] = n[d] + (!P.per[d] && cb[d] == P.p[d] - 1 ? 1 : 0);
      } else if (send) {
        x.lo[d] = o[d] > 0 ? n[d] - P.G : 0;
        x.ext[d] = o[d] > 0 ? P.G : P.G + 1;
      } else {
        x.lo[d] = o[d] < 0 ? -P.G : n[d];
        x.ext[d] = o[d] < 0 ? P.G : P.G + 1;
      }
    }
    x.offset = off;
    off += (long long)x.ext[0] * x.ext[1] * x.ext[2];
  }
  *count = m;
  if (slots) *slots = off;
  return MHD_OK;
}

// ---------------------------------------------------------------------------
// Device side
// ---------------------------------------------------------------------------
struct HaloTable {                 // a brick's boxes, by value in the kernel parameters
  int n;
  int lo[kMaxBoxes][3];
  int ext[kMaxBoxes][3];
  long long start[kMaxBoxes + 1];  // first work item (slot) of each box
  long long off[kMaxBoxes];        // first double of each box in the buffer (8 fields x its slots)
};

HaloTable make_table(const mhd_halo_box* boxes, int n) {
  HaloTable t{};
  t.n = n;
  long long s = 0;
  for (int r = 0; r < n; r++) {
    for (int d = 0; d < 3; d++) {
      t.lo[r][d] = boxes[r].lo[d];
      t.ext[r][d] = boxes[r].ext[d];
    }
    t.start[r] = s;
    t.off[r] = 8 * boxes[r].offset;
    s += (long long)boxes[r].ext[0] * boxes[r].ext[1] * boxes[r].ext[2];
  }
  t.start[n] = s;
  return t;
}

// One slot of a box: the 8 state fields, field-major within the box
// (buffer[off + q * slots_of_box + k]).  PACK reads the fields, else writes them.
template <bool PACK>
__global__ void __launch_bounds__(256) halo_kernel(Grid g, F8 S, HaloTable t, double* __restrict__ buf) {
  const long long total = t.start[t.n];
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    int r = 0;
    while (id >= t.start[r + 1]) r++;
    const long long k = id - t.start[r];
    const long long cnt = t.start[r + 1] - t.start[r];
    const int x = (int)(k % t.ext[r][0]);
    const long long rest = k / t.ext[r][0];
    const int y = (int)(rest % t.ext[r][1]);
    const int z = (int)(rest / t.ext[r][1]);
    const int c = g.at(t.lo[r][0] + x, t.lo[r][1] + y, t.lo[r][2] + z);
    double* p = buf + t.off[r] + k;
#pragma unroll
    for (int q = 0; q < 8; q++) {
      if (PACK) p[q * cnt] = S.q[q][c];
      else S.q[q][c] = p[q * cnt];
    }
  }
}

__global__ void outflow_copy_kernel(Grid g, F8 S, int d, int sides) {
  const long long total = ghost_layers_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ghost_outflow_copy_item(g, S, d, id, sides);
}
__global__ void outflow_normal_kernel(Grid g, F8 S, int d, int sides) {
  const long long total = ghost_rows_work(g, d);
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x)
    ghost_outflow_normal_item(g, S, d, id, sides);
}

// The domain's step: the least of the bricks' CFL steps (each formed by its
// cfl_exact_kernel as cfl / its largest rate), given to every brick; the
// domain's time advances by it.
__global__ void domain_dt_kernel(DevScalars* const* bsc, int nb, DevScalars* dsc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double dt = bsc[0]->dt;
  for (int b = 1; b < nb; b++) dt = fmin(dt, bsc[b]->dt);
  const double t = dsc->time + dt;
  dsc->dt = dt;
  dsc->time = t;
  for (int b = 0; b < nb; b++) {
    bsc[b]->dt = dt;
    bsc[b]->time = t;
  }
}
__global__ void domain_set_dt_kernel(DevScalars* const* bsc, int nb, DevScalars* dsc, double dt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double t = dsc->time + dt;
  dsc->dt = dt;
  dsc->time = t;
  for (int b = 0; b < nb; b++) {
    bsc[b]->dt = dt;
    bsc[b]->time = t;
  }
}

struct Copy {
  int dst;            // receiving brick
  long long dst_off;  // doubles into its receive buffer
  long long src_off;  // doubles into the sender's send buffer
  long long count;    // doubles
};

}  // namespace

struct mhd_domain {
  mhd_config cfg;
  Part part;
  int nb;
  cudaStream_t stream;
  bool own_stream;
  std::vector<mhd_ctx*> bricks;
  std::vector<int> lo, n;                 // per brick, 3 each
  std::vector<HaloTable> send, recv;
  std::vector<std::vector<Copy>> copies;  // per sending brick
  std::vector<long long> send_base, recv_base;
  std::vector<long long> send_used, recv_used;  // doubles of each brick's region
  std::vector<int> outflow_sides;         // per brick and axis: bit 0 low, bit 1 high
  double* sendbuf = nullptr;
  double* recvbuf = nullptr;
  long long halo_doubles = 0;             // doubles moved per exchange
  DevScalars* dsc = nullptr;
  DevScalars** bsc = nullptr;             // device array of the bricks' scalars
  cudaGraphExec_t graph;
  bool graph_ready = false;
  bool has_state = false;
  long long own_launches = 0, replayed = 0;
  int launches_per_step = 0;
};

namespace {

long long total_launches(const mhd_domain* D) {
  long long s = D->own_launches + D->replayed;
  for (const mhd_ctx* c : D->bricks) s += c->launches;
  return s;
}

// The ghost shells of register r of every brick: pack, exchange, unpack, then
// the outflow sides in axis order (as the undivided grid fills periodic axes
// before outflow ones, each pass over the full padded transverse range).
void domain_fill(mhd_domain* D, int r) {
  for (int b = 0; b < D->nb; b++) {
    mhd_ctx* c = D->bricks[b];
    const HaloTable& t = D->send[b];
    if (!t.n) continue;
    halo_kernel<true><<<blocks_for(t.start[t.n], 256), 256, 0, D->stream>>>(c->g, c->U[r], t,
                                                                            D->sendbuf + D->send_base[b]);
    D->own_launches++;
  }
  for (int b = 0; b < D->nb; b++)
    for (const Copy& x : D->copies[b])
      cudaMemcpyAsync(D->recvbuf + D->recv_base[x.dst] + x.dst_off, D->sendbuf + D->send_base[b] + x.src_off,
                      x.count * sizeof(double), cudaMemcpyDeviceToDevice, D->stream);
  for (int b = 0; b < D->nb; b++) {
    mhd_ctx* c = D->bricks[b];
    const HaloTable& t = D->recv[b];
    if (t.n) {
      halo_kernel<false><<<blocks_for(t.start[t.n], 256), 256, 0, D->stream>>>(c->g, c->U[r], t,
                                                                               D->recvbuf + D->recv_base[b]);
      D->own_launches++;
    }
    const Grid& g = c->g;
    for (int d = 0; d < g.ndim; d++) {
      const int sides = D->outflow_sides[3 * b + d];
      if (!sides) continue;
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      const long long rows = (long long)(g.hi(t1) - g.lo(t1) + 1) * (g.hi(t2) - g.lo(t2) + 1);
      outflow_copy_kernel<<<blocks_for(rows * (2 * g.G + 1), 256), 256, 0, D->stream>>>(g, c->U[r], d, sides);
      outflow_normal_kernel<<<blocks_for(rows, 128), 128, 0, D->stream>>>(g, c->U[r], d, sides);
      D->own_launches += 2;
    }
  }
}

// Stage s: the registers of run_stage (input U[0], U[1], U[2]; output U[1],
// then U[0] or U[2]), every brick's phase issued before the next phase.
void domain_stage(mhd_domain* D, int s, bool cfl) {
  const int rk = D->cfg.rk;
  const int rs = s;
  const int ro = s == 0 ? 1 : ((rk == 2 || s == 2) ? 0 : 2);
  domain_fill(D, rs);
  for (mhd_ctx* c : D->bricks) prim(c, c->U[rs], cfl, s > 0);
  if (cfl) {
    domain_dt_kernel<<<1, 32, 0, D->stream>>>(D->bsc, D->nb, D->dsc);
    D->own_launches++;
  }
  for (mhd_ctx* c : D->bricks) {
    sweeps(c, c->U[rs]);
    emf(c, c->U[rs]);
    ct_rk(c, c->U[0], c->U[rs], c->U[ro], stage_mode(rk, s));
  }
}

void domain_run_step(mhd_domain* D, bool device_dt) {
  for (int s = 0; s < D->cfg.rk; s++) domain_stage(D, s, device_dt && s == 0);
}

// Box copies between a whole-grid array in the boundary layout (extents E,
// host or device) and brick b's padded field q: the brick's interior of slot
// q (faces [0, n] along the face axis when upper = true, else [0, n - 1]).
int copy_brick_field(mhd_domain* D, int b, int q, const double* in, double* out, bool upper_face) {
  mhd_ctx* c = D->bricks[b];
  const Grid& g = c->g;
  int E[3], e[3];
  for (int d = 0; d < 3; d++) {
    E[d] = D->part.N[d];
    e[d] = D->n[3 * b + d];
  }
  if (q >= 5 && q - 5 < g.ndim) {
    E[q - 5] += 1;
    if (upper_face) e[q - 5] += 1;
  }
  const int* lo = &D->lo[3 * b];
  cudaMemcpy3DParms p{};
  cudaPitchedPtr whole = make_cudaPitchedPtr(in ? (void*)in : (void*)out, (size_t)E[0] * 8, E[0], E[1]);
  cudaPitchedPtr padded = make_cudaPitchedPtr((void*)c->U[0].q[q], (size_t)g.ext[0] * 8, g.ext[0], g.ext[1]);
  const int Gz = g.ndim == 3 ? g.G : 0;
  cudaPos wpos = make_cudaPos((size_t)lo[0] * 8, lo[1], lo[2]);
  cudaPos ppos = make_cudaPos((size_t)g.G * 8, g.G, Gz);
  if (in) {
    p.srcPtr = whole;
    p.srcPos = wpos;
    p.dstPtr = padded;
    p.dstPos = ppos;
  } else {
    p.srcPtr = padded;
    p.srcPos = ppos;
    p.dstPtr = whole;
    p.dstPos = wpos;
  }
  p.extent = make_cudaExtent((size_t)e[0] * 8, e[1], e[2]);
  p.kind = cudaMemcpyDefault;
  CK(cudaMemcpy3DAsync(&p, D->stream));
  return MHD_OK;
}

void free_domain(mhd_domain* D) {
  if (D->stream) cudaStreamSynchronize(D->stream);
  if (D->graph_ready) cudaGraphExecDestroy(D->graph);
  for (mhd_ctx* c : D->bricks) mhd_destroy(c);
  cudaFree(D->sendbuf);
  cudaFree(D->recvbuf);
  cudaFree(D->dsc);
  cudaFree(D->bsc);
  if (D->own_stream) cudaStreamDestroy(D->stream);
  delete D;
}

}  // namespace

extern "C" {

int mhd_domain_brick(const mhd_config* cfg, const int parts[3], int brick, int lo[3], int n[3]) {
  Part P;
  int rc = make_part(cfg, parts, P);
  if (rc) return rc;
  if (brick < 0 || brick >= nbricks(P) || !lo || !n) return MHD_ERR_ARG;
  brick_box(P, brick, lo, n);
  return MHD_OK;
}

int mhd_domain_halo(const mhd_config* cfg, const int parts[3], int brick, int send, mhd_halo_box* boxes,
                    int max_boxes, int* nboxes) {
  Part P;
  int rc = make_part(cfg, parts, P);
  if (rc) return rc;
  if (brick < 0 || brick >= nbricks(P) || !boxes || !nboxes || max_boxes < 0) return MHD_ERR_ARG;
  return halo_boxes(P, brick, send != 0, boxes, max_boxes, nboxes, nullptr);
}

int mhd_domain_create(const mhd_config* cfg, const int parts[3], mhd_domain** out) {
  if (!out) return MHD_ERR_ARG;
  *out = nullptr;
  Part P;
  int rc = make_part(cfg, parts, P);
  if (rc) return rc;
  mhd_domain* D = new (std::nothrow) mhd_domain();
  if (!D) return MHD_ERR_OOM;
  D->cfg = *cfg;
  D->part = P;
  D->nb = nbricks(P);
  if (cfg->stream) {
    D->stream = (cudaStream_t)cfg->stream;
  } else {
    if (cudaStreamCreate(&D->stream) != cudaSuccess) {
      delete D;
      return MHD_ERR_CUDA;
    }
    D->own_stream = true;
  }
  const Grid whole = make_grid(cfg);
  D->lo.resize(3 * D->nb);
  D->n.resize(3 * D->nb);
  D->outflow_sides.assign(3 * D->nb, 0);
  std::vector<std::vector<mhd_halo_box>> sb(D->nb), rb(D->nb);
  long long send_total = 0, recv_total = 0;
  D->send_base.resize(D->nb);
  D->recv_base.resize(D->nb);
  D->send_used.resize(D->nb);
  D->recv_used.resize(D->nb);
  for (int b = 0; b < D->nb; b++) {
    int* lo = &D->lo[3 * b];
    int* n = &D->n[3 * b];
    brick_box(P, b, lo, n);
    mhd_config bc = *cfg;
    bc.nx = n[0];
    bc.ny = n[1];
    bc.nz = n[2];
    for (int d = 0; d < cfg->ndim; d++) {
      bc.x0[d] = cfg->x0[d] + lo[d] * whole.dx[d];
      bc.x1[d] = cfg->x0[d] + (lo[d] + n[d]) * whole.dx[d];
      int c[3];
      brick_coord(P, b, c);
      if (!P.per[d]) D->outflow_sides[3 * b + d] = (c[d] == 0 ? 1 : 0) | (c[d] == P.p[d] - 1 ? 2 : 0);
    }
    bc.stream = D->stream;
    mhd_ctx* ctx = nullptr;
    rc = mhd_create(&bc, &ctx);
    if (rc) {
      free_domain(D);
      return rc;
    }
    D->bricks.push_back(ctx);
    // the whole grid's spacing, to the bit (the brick's own bounds may round differently)
    for (int d = 0; d < 3; d++) {
      ctx->g.dx[d] = whole.dx[d];
      ctx->g.idx[d] = whole.idx[d];
    }
    sb[b].resize(kMaxBoxes);
    rb[b].resize(kMaxBoxes);
    int ns = 0, nr = 0;
    long long ss = 0, rs = 0;
    halo_boxes(P, b, true, sb[b].data(), kMaxBoxes, &ns, &ss);
    halo_boxes(P, b, false, rb[b].data(), kMaxBoxes, &nr, &rs);
    sb[b].resize(ns);
    rb[b].resize(nr);
    D->send.push_back(make_table(sb[b].data(), ns));
    D->recv.push_back(make_table(rb[b].data(), nr));
    // each brick's region of a buffer is a guarded block of one field
    D->send_base[b] = send_total + kGuardWords;
    D->recv_base[b] = recv_total + kGuardWords;
    D->send_used[b] = 8 * ss;
    D->recv_used[b] = 8 * rs;
    send_total += guard_block_words(1, guard_stride(8 * ss));
    recv_total += guard_block_words(1, guard_stride(8 * rs));
  }
  // each box sent in direction o lands in the peer's box received from direction -o
  D->copies.resize(D->nb);
  for (int b = 0; b < D->nb; b++)
    for (const mhd_halo_box& s : sb[b]) {
      const mhd_halo_box* r = nullptr;
      for (const mhd_halo_box& x : rb[s.peer])
        if (x.dir[0] == -s.dir[0] && x.dir[1] == -s.dir[1] && x.dir[2] == -s.dir[2]) r = &x;
      const long long cnt = 8LL * s.ext[0] * s.ext[1] * s.ext[2];
      if (!r || 8LL * r->ext[0] * r->ext[1] * r->ext[2] != cnt) {
        free_domain(D);
        return MHD_ERR_ARG;
      }
      D->copies[b].push_back({s.peer, 8 * r->offset, 8 * s.offset, cnt});
      D->halo_doubles += cnt;
    }
  bool ok = cudaMalloc(&D->sendbuf, std::max<long long>(send_total, 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&D->recvbuf, std::max<long long>(recv_total, 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&D->dsc, sizeof(DevScalars)) == cudaSuccess &&
            cudaMalloc(&D->bsc, D->nb * sizeof(DevScalars*)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_domain(D);
    return MHD_ERR_OOM;
  }
  for (int b = 0; b < D->nb && ok; b++)
    ok = guard_fill(D->stream, D->sendbuf + D->send_base[b] - kGuardWords, 1, guard_stride(D->send_used[b]),
                    D->send_used[b]) == MHD_OK &&
         guard_fill(D->stream, D->recvbuf + D->recv_base[b] - kGuardWords, 1, guard_stride(D->recv_used[b]),
                    D->recv_used[b]) == MHD_OK;
  if (!ok) {
    free_domain(D);
    return MHD_ERR_CUDA;
  }
  std::vector<DevScalars*> ptrs(D->nb);
  for (int b = 0; b < D->nb; b++) ptrs[b] = D->bricks[b]->sc;
  DevScalars h;
  reset_scalars_host(&h);
  if (cudaMemcpyAsync(D->bsc, ptrs.data(), D->nb * sizeof(DevScalars*), cudaMemcpyHostToDevice, D->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(D->dsc, &h, sizeof(h), cudaMemcpyHostToDevice, D->stream) != cudaSuccess ||
      cudaStreamSynchronize(D->stream) != cudaSuccess) {
    free_domain(D);
    return MHD_ERR_CUDA;
  }
  *out = D;
  return MHD_OK;
}

int mhd_domain_destroy(mhd_domain* D) {
  if (!D) return MHD_OK;
  free_domain(D);
  return MHD_OK;
}

int mhd_domain_set_conserved(mhd_domain* D, int mem, const double* const* U, const double* const* B) {
  if (!D || !U || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  for (int q = 0; q < 8; q++)
    if (!(q < 5 ? U[q] : B[q - 5])) return MHD_ERR_ARG;
  for (int b = 0; b < D->nb; b++) {
    for (int q = 0; q < 8; q++) {
      int rc = copy_brick_field(D, b, q, q < 5 ? U[q] : B[q - 5], nullptr, true);
      if (rc) return rc;
    }
    mhd_ctx* c = D->bricks[b];
    CK(cudaMemcpyAsync(c->sc, reset_scalars_source(), sizeof(DevScalars), cudaMemcpyHostToDevice, D->stream));
    c->has_state = true;
  }
  CK(cudaMemcpyAsync(D->dsc, reset_scalars_source(), sizeof(DevScalars), cudaMemcpyHostToDevice, D->stream));
  // the copies from pageable host memory are staged before the call returns,
  // device and pinned ones run in stream order
  D->has_state = true;
  return MHD_OK;
}

int mhd_domain_get_conserved(mhd_domain* D, int mem, double* const* U, double* const* B) {
  if (!D || !U || !B || (mem != MHD_MEM_HOST && mem != MHD_MEM_DEVICE)) return MHD_ERR_ARG;
  if (!D->has_state) return MHD_ERR_STATE;
  for (int q = 0; q < 8; q++)
    if (!(q < 5 ? U[q] : B[q - 5])) return MHD_ERR_ARG;
  domain_fill(D, 0);  // a periodic axis's last face, as the undivided grid writes it
  CK(cudaGetLastError());
  int c3[3];
  for (int b = 0; b < D->nb; b++) {
    brick_coord(D->part, b, c3);
    for (int q = 0; q < 8; q++) {
      // the upper face of a face axis belongs to the next brick, except on the last one
      const bool upper = q >= 5 && q - 5 < D->cfg.ndim && c3[q - 5] == D->part.p[q - 5] - 1;
      int rc = copy_brick_field(D, b, q, nullptr, q < 5 ? U[q] : B[q - 5], upper);
      if (rc) return rc;
    }
  }
  return mhd_domain_status(D, nullptr);
}

int mhd_domain_cfl_dt(mhd_domain* D, double* dt_out) {
  if (!D || !dt_out) return MHD_ERR_ARG;
  if (!D->has_state) return MHD_ERR_STATE;
  std::vector<DevScalars> before(D->nb);
  DevScalars dbefore;
  CK(cudaStreamSynchronize(D->stream));
  for (int b = 0; b < D->nb; b++)
    CK(cudaMemcpyAsync(&before[b], D->bricks[b]->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, D->stream));
  CK(copy_sync(&dbefore, D->dsc, sizeof(dbefore), cudaMemcpyDeviceToHost, D->stream));
  domain_fill(D, 0);
  for (mhd_ctx* c : D->bricks) prim(c, c->U[0], true);
  domain_dt_kernel<<<1, 32, 0, D->stream>>>(D->bsc, D->nb, D->dsc);
  D->own_launches++;
  CK(cudaGetLastError());
  DevScalars after;
  CK(copy_sync(&after, D->dsc, sizeof(after), cudaMemcpyDeviceToHost, D->stream));
  *dt_out = after.dt;
  // evaluating dt does not advance the time: restore dt and time
  int st = MHD_OK;
  for (int b = 0; b < D->nb; b++) {
    DevScalars a;
    CK(copy_sync(&a, D->bricks[b]->sc, sizeof(a), cudaMemcpyDeviceToHost, D->stream));
    if (a.status) st = a.status;
    a.dt = before[b].dt;
    a.time = before[b].time;
    CK(copy_sync(D->bricks[b]->sc, &a, sizeof(a), cudaMemcpyHostToDevice, D->stream));
  }
  after.dt = dbefore.dt;
  after.time = dbefore.time;
  CK(copy_sync(D->dsc, &after, sizeof(after), cudaMemcpyHostToDevice, D->stream));
  return st;
}

int mhd_domain_step(mhd_domain* D, double dt) {
  if (!D || !(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_ARG;
  if (!D->has_state) return MHD_ERR_STATE;
  domain_set_dt_kernel<<<1, 32, 0, D->stream>>>(D->bsc, D->nb, D->dsc, dt);
  D->own_launches++;
  domain_run_step(D, false);
  CK(cudaGetLastError());
  return MHD_OK;
}

int mhd_domain_advance(mhd_domain* D, int nsteps) {
  if (!D || nsteps < 0) return MHD_ERR_ARG;
  if (!D->has_state) return MHD_ERR_STATE;
  if (nsteps == 0) return MHD_OK;
  if (!D->graph_ready) {
    std::vector<long long> saved(D->nb);
    for (int b = 0; b < D->nb; b++) saved[b] = D->bricks[b]->launches;
    const long long own = D->own_launches, before = total_launches(D);
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(D->stream, cudaStreamCaptureModeThreadLocal));
    domain_run_step(D, true);
    cudaError_t e = cudaStreamEndCapture(D->stream, &graph);
    if (e != cudaSuccess) return cuda_err(e);
    e = cudaGraphInstantiate(&D->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_err(e);
    D->graph_ready = true;
    D->launches_per_step = (int)(total_launches(D) - before);
    for (int b = 0; b < D->nb; b++) D->bricks[b]->launches = saved[b];
    D->own_launches = own;
  }
  for (int s = 0; s < nsteps; s++) {
    CK(cudaGraphLaunch(D->graph, D->stream));
    D->replayed += D->launches_per_step;
  }
  return MHD_OK;
}

int mhd_domain_get_time(mhd_domain* D, double* t_out) {
  if (!D || !t_out) return MHD_ERR_ARG;
  DevScalars h;
  CK(copy_sync(&h, D->dsc, sizeof(h), cudaMemcpyDeviceToHost, D->stream));
  *t_out = h.time;
  return MHD_OK;
}

int mhd_domain_status(mhd_domain* D, long long* bad_cell) {
  if (!D) return MHD_ERR_ARG;
  CK(cudaStreamSynchronize(D->stream));
  int st = MHD_OK;
  long long best = LLONG_MAX;
  const long long NX = D->part.N[0], NY = D->part.N[1];
  for (int b = 0; b < D->nb; b++) {
    DevScalars h;
    CK(copy_sync(&h, D->bricks[b]->sc, sizeof(h), cudaMemcpyDeviceToHost, D->stream));
    if (!h.status) continue;
    st = h.status;
    // brick-local flat index k*ny*nx + j*nx + i of the brick's interior -> the whole grid's
    const int* lo = &D->lo[3 * b];
    const int* n = &D->n[3 * b];
    const long long i = h.bad_cell % n[0], j = (h.bad_cell / n[0]) % n[1], k = h.bad_cell / ((long long)n[0] * n[1]);
    best = std::min(best, ((k + lo[2]) * NY + (j + lo[1])) * NX + (i + lo[0]));
    h.status = 0;
    h.bad_cell = LLONG_MAX;
    CK(copy_sync(D->bricks[b]->sc, &h, sizeof(h), cudaMemcpyHostToDevice, D->stream));
  }
  if (bad_cell) *bad_cell = st ? best : -1;
  return st;
}

int mhd_domain_counters(mhd_domain* D, long long* recon_fallbacks, long long* pressure_floors) {
  if (!D) return MHD_ERR_ARG;
  long long f = 0, p = 0;
  for (mhd_ctx* c : D->bricks) {
    long long a = 0, b = 0;
    int rc = mhd_counters(c, &a, &b);
    if (rc) return rc;
    f += a;
    p += b;
  }
  if (recon_fallbacks) *recon_fallbacks = f;
  if (pressure_floors) *pressure_floors = p;
  return MHD_OK;
}

int mhd_domain_set_seglen(mhd_domain* D, int seglen) {
  if (!D || seglen < 1) return MHD_ERR_ARG;
  for (mhd_ctx* c : D->bricks) {
    int rc = mhd_set_seglen(c, seglen);
    if (rc) return rc;
  }
  if (D->graph_ready) {
    cudaGraphExecDestroy(D->graph);
    D->graph_ready = false;
  }
  return MHD_OK;
}

long long mhd_domain_launch_count(const mhd_domain* D) { return D ? total_launches(D) : 0; }

long long mhd_domain_halo_bytes(const mhd_domain* D) { return D ? D->halo_doubles * (long long)sizeof(double) : 0; }

}  // extern "C"

int mhd_domain_check_guards(mhd_domain* D, int* brick, int* field, long long* word) {
  if (!D || !brick || !field || !word) return MHD_ERR_ARG;
  for (int b = 0; b < D->nb; b++) {
    int rc = mhd_check_guards(D->bricks[b], field, word);
    if (rc == MHD_ERR_GUARD) *brick = b;
    if (rc) return rc;
  }
  // the bricks' regions of the send buffer, then of the receive buffer
  for (int which = 0; which < 2; which++) {
    std::vector<const double*> base(D->nb);
    std::vector<int> nf(D->nb, 1);
    std::vector<long long> stride(D->nb);
    const std::vector<long long>& used = which ? D->recv_used : D->send_used;
    for (int b = 0; b < D->nb; b++) {
      base[b] = (which ? D->recvbuf + D->recv_base[b] : D->sendbuf + D->send_base[b]) - kGuardWords;
      stride[b] = guard_stride(used[b]);
    }
    int rc = guard_check_blocks(D->stream, D->nb, base.data(), nf.data(), stride.data(), used.data(), brick, field,
                                word);
    if (rc == MHD_ERR_GUARD) *field = which ? MHD_GUARD_RECV : MHD_GUARD_SEND;
    if (rc) return rc;
  }
  *brick = *field = -1;
  *word = -1;
  return MHD_OK;
}
