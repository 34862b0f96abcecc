// The assembled operator w = M Q^T A_L Q M u (Sec. 2.2) on vectors in host
// memory, with the transfers pipelined against the arithmetic.
//
// Unique nodes are numbered plane by plane in z (g = I + nx (J + ny K)), so a
// slab of element layers ez in [z0, z1) reads u only on the lattice planes
// K in [z0 N, z1 N] and writes w only there. The elements are cut into such
// slabs; three streams run the pipeline: the copy-in stream brings the planes
// the next slab needs, the caller's stream applies the operator to a slab as
// soon as its planes have arrived, and the copy-out stream returns the planes
// a finished slab completes (a plane shared with the next slab waits for it).
// Element sub-ranges reuse the ordinary kernels through a copy of the mesh
// descriptor whose per-element arrays start at the slab's first element.
#include <algorithm>
#include <vector>

#include "sem_internal.h"

namespace {

struct IoStreams {
  cudaStream_t in = nullptr, out = nullptr;
  std::vector<cudaEvent_t> ev;
  ~IoStreams() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (in) cudaStreamDestroy(in);
    if (out) cudaStreamDestroy(out);
  }
  cudaEvent_t make() {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    ev.push_back(e);
    return e;
  }
};

// a descriptor of elements [e0, e1) of m: the same unique numbering, shifted per-element arrays
sem_mesh sub_range(const sem_mesh *m, int64_t e0, int64_t e1) {
  sem_mesh s = *m;
  const int64_t n3 = m->n3;
  s.E = e1 - e0;
  s.n_local = s.E * n3;
  s.X = m->X + e0 * n3;
  s.Y = m->Y + e0 * n3;
  s.Z = m->Z + e0 * n3;
  s.G = m->G + e0 * 6 * n3;
  s.Gdf = m->Gdf + e0 * 6 * n3;
  s.B = m->B + e0 * n3;
  s.Bdf = m->Bdf + e0 * n3;
  s.l2g = m->l2g + e0 * n3;
  s.l2gm = m->l2gm + e0 * n3;
  s.det_w = nullptr;
  s.K1 = nullptr;
  s.K1df = nullptr;
  return s;
}

}  // namespace

extern "C" int sem_ax_assembled_host(const sem_mesh *m, double h1, double h2, const double *u_host, double *w_host,
                                     int precision, double *u_dev, double *w_dev, int nchunks, void *stream) {
  SemRange nvtx_range("sem_ax_assembled_host");
  if (m && m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host: needs the whole box, not a partition's slab mesh");
  if (!m || !u_host || !w_host || !u_dev || !w_dev)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host: NULL argument");
  if ((((uintptr_t)u_dev) | ((uintptr_t)w_dev)) & 7 || u_dev == w_dev)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host: misaligned or overlapping device vectors");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host: unknown precision");
  int dev = -1;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host: the mesh's device must be current");
  cudaStream_t st = as_stream(stream);
  const int N = m->N, nelz = m->nel[2];
  const bool pz = m->periodic[2] != 0;
  const int64_t nx = (int64_t)m->nel[0] * N + (m->periodic[0] ? 0 : 1);
  const int64_t ny = (int64_t)m->nel[1] * N + (m->periodic[1] ? 0 : 1);
  const int64_t nzp = (int64_t)nelz * N + (pz ? 0 : 1);
  const int64_t plane = nx * ny;
  const int64_t layer = (int64_t)m->nel[0] * m->nel[1];
  // element matrices (N = 1) and deterministic assembly work on whole meshes only
  int nc = (nchunks <= 0) ? 8 : nchunks;
  if (m->K1 || m->det_w) nc = 1;
  nc = std::max(1, std::min(nc, nelz));

  IoStreams io;
  SEM_CUDA(cudaStreamCreateWithFlags(&io.in, cudaStreamNonBlocking));
  SEM_CUDA(cudaStreamCreateWithFlags(&io.out, cudaStreamNonBlocking));
  cudaEvent_t start = io.make(), done_out = io.make();
  if (!start || !done_out) return sem_fail(SEM_ERR_CUDA, "sem_ax_assembled_host: cudaEventCreate");
  // the side streams start after everything already queued on the caller's stream
  SEM_CUDA(cudaEventRecord(start, st));
  SEM_CUDA(cudaStreamWaitEvent(io.in, start, 0));
  SEM_CUDA(cudaStreamWaitEvent(io.out, start, 0));
  SEM_CUDA(cudaMemsetAsync(w_dev, 0, sizeof(double) * m->n_unique, st));

  int64_t in_hi = 0;  // planes [0, in_hi) copied in so far
  for (int c = 0; c < nc; ++c) {
    const int z0 = (int)((int64_t)c * nelz / nc), z1 = (int)((int64_t)(c + 1) * nelz / nc);
    // copy in the planes up to z1 N (the wrapped top plane of a periodic z is plane 0, already in)
    const int64_t need = std::min<int64_t>((int64_t)z1 * N + 1, nzp);
    if (need > in_hi) {
      SEM_CUDA(cudaMemcpyAsync(u_dev + in_hi * plane, u_host + in_hi * plane, sizeof(double) * (need - in_hi) * plane,
                               cudaMemcpyHostToDevice, io.in));
      in_hi = need;
    }
    cudaEvent_t ev_in = io.make(), ev_comp = io.make();
    if (!ev_in || !ev_comp) return sem_fail(SEM_ERR_CUDA, "sem_ax_assembled_host: cudaEventCreate");
    SEM_CUDA(cudaEventRecord(ev_in, io.in));
    SEM_CUDA(cudaStreamWaitEvent(st, ev_in, 0));
    if (nc == 1) {
      if (int rc = sem_launch_ax_assembled(m, h1, h2, u_dev, w_dev, nullptr, precision, st)) return rc;
    } else {
      const sem_mesh sub = sub_range(m, (int64_t)z0 * layer, (int64_t)z1 * layer);
      if (int rc = sem_launch_ax_assembled(&sub, h1, h2, u_dev, w_dev, nullptr, precision, st)) return rc;
    }
    SEM_CUDA(cudaEventRecord(ev_comp, st));
    SEM_CUDA(cudaStreamWaitEvent(io.out, ev_comp, 0));
    // planes this slab completes: [z0 N, z1 N), or up to the end for the last slab;
    // plane 0 of a periodic z also receives the last slab, so it leaves last
    int64_t lo = (int64_t)z0 * N, hi = (c == nc - 1) ? nzp : (int64_t)z1 * N;
    if (pz && z0 == 0) lo = 1;
    if (hi > lo)
      SEM_CUDA(cudaMemcpyAsync(w_host + lo * plane, w_dev + lo * plane, sizeof(double) * (hi - lo) * plane,
                               cudaMemcpyDeviceToHost, io.out));
  }
  if (pz) SEM_CUDA(cudaMemcpyAsync(w_host, w_dev, sizeof(double) * plane, cudaMemcpyDeviceToHost, io.out));
  SEM_CUDA(cudaEventRecord(done_out, io.out));
  SEM_CUDA(cudaStreamWaitEvent(st, done_out, 0));
  SEM_CUDA(cudaStreamSynchronize(st));
  return SEM_OK;
}

// Several independent applications on host vectors, pipelined across the
// applications instead of within one: the copy-in of application k + 1, the
// operator of application k and the copy-out of application k - 1 run at the
// same time, each copy moving one whole vector (cutting a vector into chunks
// costs link throughput). Device vectors are double-buffered: application k
// uses u_dev2 + (k & 1) n_unique and w_dev2 + (k & 1) n_unique.
extern "C" int sem_ax_assembled_host_batch(const sem_mesh *m, double h1, double h2, int nsteps,
                                           const double *const *u_host, double *const *w_host, int precision,
                                           double *u_dev2, double *w_dev2, void *stream) {
  SemRange nvtx_range("sem_ax_assembled_host_batch");
  if (m && m->slab) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host_batch: needs the whole box, not a partition's slab mesh");
  if (!m || !u_host || !w_host || !u_dev2 || !w_dev2 || nsteps < 0)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host_batch: NULL argument or negative count");
  for (int k = 0; k < nsteps; ++k)
    if (!u_host[k] || !w_host[k]) return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host_batch: NULL host vector");
  if ((((uintptr_t)u_dev2) | ((uintptr_t)w_dev2)) & 7 || u_dev2 == w_dev2)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host_batch: misaligned or overlapping device vectors");
  if (precision != SEM_PREC_FP64 && precision != SEM_PREC_DF64)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host_batch: unknown precision");
  int dev = -1;
  SEM_CUDA(cudaGetDevice(&dev));
  if (dev != m->device)
    return sem_fail(SEM_ERR_INVALID_ARG, "sem_ax_assembled_host_batch: the mesh's device must be current");
  if (nsteps == 0) return SEM_OK;
  cudaStream_t st = as_stream(stream);
  const int64_t nU = m->n_unique;
  const size_t bytes = sizeof(double) * (size_t)nU;

  IoStreams io;
  SEM_CUDA(cudaStreamCreateWithFlags(&io.in, cudaStreamNonBlocking));
  SEM_CUDA(cudaStreamCreateWithFlags(&io.out, cudaStreamNonBlocking));
  cudaEvent_t start = io.make();
  if (!start) return sem_fail(SEM_ERR_CUDA, "sem_ax_assembled_host_batch: cudaEventCreate");
  SEM_CUDA(cudaEventRecord(start, st));
  SEM_CUDA(cudaStreamWaitEvent(io.in, start, 0));
  SEM_CUDA(cudaStreamWaitEvent(io.out, start, 0));
  // per application: copy-in done, operator done, copy-out done
  std::vector<cudaEvent_t> ev_in(nsteps), ev_op(nsteps), ev_out(nsteps);
  for (int k = 0; k < nsteps; ++k) {
    ev_in[k] = io.make();
    ev_op[k] = io.make();
    ev_out[k] = io.make();
    if (!ev_in[k] || !ev_op[k] || !ev_out[k]) return sem_fail(SEM_ERR_CUDA, "sem_ax_assembled_host_batch: cudaEventCreate");
  }
  for (int k = 0; k < nsteps; ++k) {
    double *ub = u_dev2 + (size_t)(k & 1) * nU;
    double *wb = w_dev2 + (size_t)(k & 1) * nU;
    // copy-in: u buffer free once application k - 2's operator has read it
    if (k >= 2) SEM_CUDA(cudaStreamWaitEvent(io.in, ev_op[k - 2], 0));
    SEM_CUDA(cudaMemcpyAsync(ub, u_host[k], bytes, cudaMemcpyHostToDevice, io.in));
    SEM_CUDA(cudaEventRecord(ev_in[k], io.in));
    // operator: after its copy-in, and after application k - 2's result left w buffer
    SEM_CUDA(cudaStreamWaitEvent(st, ev_in[k], 0));
    if (k >= 2) SEM_CUDA(cudaStreamWaitEvent(st, ev_out[k - 2], 0));
    SEM_CUDA(cudaMemsetAsync(wb, 0, bytes, st));
    if (int rc = sem_launch_ax_assembled(m, h1, h2, ub, wb, nullptr, precision, st)) return rc;
    SEM_CUDA(cudaEventRecord(ev_op[k], st));
    // copy-out
    SEM_CUDA(cudaStreamWaitEvent(io.out, ev_op[k], 0));
    SEM_CUDA(cudaMemcpyAsync(w_host[k], wb, bytes, cudaMemcpyDeviceToHost, io.out));
    SEM_CUDA(cudaEventRecord(ev_out[k], io.out));
  }
  SEM_CUDA(cudaStreamWaitEvent(st, ev_out[nsteps - 1], 0));
  SEM_CUDA(cudaStreamSynchronize(st));
  return SEM_OK;
}
