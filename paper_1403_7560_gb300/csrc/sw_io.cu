// Asynchronous host I/O of a lattice's state, overlapping with its sweeps.
//
// The paper has no counterpart: it times sweeps on a resident lattice.  A
// serving loop that streams states in and results out needs the transfers
// off the sweep's critical path.  Uploads run on their own stream into a
// staging buffer that is swapped with the state buffer once the upload is
// done (kernels launched afterwards read the new state); downloads copy the
// state buffer itself to the host on a second stream, so the sweeps go on
// while the download runs (they only read the buffer until the next flip,
// and the flip waits for the copy).  Events order the three streams:
//   upload k:   io_in waits ev_in_free (the buffer it fills is no longer
//               read) and, if the buffer was downloaded since its last
//               write, that download; copies, records ev_in_done; the
//               compute stream waits ev_in_done, the buffers are swapped,
//               ev_in_free is recorded.
//   download k: the compute stream records ev_state (the state is final);
//               io_out waits for it, copies the state buffer to the host and
//               records ev_down of that buffer.  The next write of the
//               buffer, on any stream, first waits for ev_down
//               (guard_state_write).
//   record:     the compute stream records ev_rec once the record is final;
//               io_out waits ev_rec and copies it (small copies issued on
//               the compute stream would queue behind a download on the
//               same copy engine and stall the sweeps).
#include <string>
#include <utility>

#include "../../include/sw.h"
#include "sw_internal.h"

namespace {

int io_fail(int code, const std::string& msg) {
  swgb::set_last_error(msg);
  return code;
}

int io_cuda(cudaError_t e, const char* what) {
  return io_fail(SW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t ensure_io(sw_handle* h) {
  if (h->io_in) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&h->io_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->io_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = swgb::dev_alloc(&h->stage_in, h->spin_bytes, h->stream);
  // the copy streams use the buffers: order them after the allocations
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  cudaEvent_t* evs[6] = {&h->ev_in_done, &h->ev_in_free, &h->ev_state, &h->ev_rec, &h->ev_down[0], &h->ev_down[1]};
  for (cudaEvent_t* ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    swgb::release_io(h);
    return e;
  }
  h->io_buf[0] = h->lat.spins;
  h->io_buf[1] = h->stage_in;
  return e;
}

int check_io_args(sw_handle* h, const void* host, size_t bytes) {
  if (!h || !host) return io_fail(SW_ERR_BAD_ARG, "NULL argument");
  if (bytes != h->spin_bytes) return io_fail(SW_ERR_BAD_ARG, "bytes != sw_spin_bytes");
  if (h->batch) return io_fail(SW_ERR_BAD_ARG, "asynchronous I/O is not available for a lattice in a batch");
  return SW_OK;
}

}  // namespace

cudaError_t swgb::guard_state_write(sw_handle* h, const void* buf, cudaStream_t st) {
  for (int i = 0; i < 2; ++i) {
    if (!h->down_wait[i] || buf != h->io_buf[i]) continue;
    // later writes of the buffer are ordered after this one: on st itself,
    // or on the other stream through the upload/swap events
    h->down_wait[i] = false;
    return cudaStreamWaitEvent(st, h->ev_down[i], 0);
  }
  return cudaSuccess;
}

cudaError_t swgb::wait_io(sw_handle* h) {
  cudaError_t e = cudaSuccess;
  if (h->io_in) e = cudaStreamSynchronize(h->io_in);
  if (e == cudaSuccess && h->io_out) e = cudaStreamSynchronize(h->io_out);
  if (e == cudaSuccess) h->down_wait[0] = h->down_wait[1] = false;
  return e;
}

void swgb::release_io(sw_handle* h) {
  if (h->io_in) cudaStreamSynchronize(h->io_in);
  if (h->io_out) cudaStreamSynchronize(h->io_out);
  cudaEvent_t evs[6] = {h->ev_in_done, h->ev_in_free, h->ev_state, h->ev_rec, h->ev_down[0], h->ev_down[1]};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  h->ev_in_done = h->ev_in_free = h->ev_state = h->ev_rec = h->ev_down[0] = h->ev_down[1] = nullptr;
  swgb::dev_free(h->stage_in, h->stream);
  h->stage_in = nullptr;
  h->io_buf[0] = h->io_buf[1] = nullptr;
  h->down_wait[0] = h->down_wait[1] = false;
  if (h->io_in) cudaStreamDestroy(h->io_in);
  if (h->io_out) cudaStreamDestroy(h->io_out);
  h->io_in = h->io_out = nullptr;
  h->in_free_set = false;
}

extern "C" {

int sw_set_spins_async(sw_handle* h, const void* host, size_t bytes) {
  int rc = check_io_args(h, host, bytes);
  if (rc != SW_OK) return rc;
  cudaError_t e = ensure_io(h);
  if (e != cudaSuccess) return io_cuda(e, "asynchronous I/O setup");
  // the pending measurement reads the state being replaced
  e = swgb::flush_pending(h);
  if (e == cudaSuccess && h->in_free_set) e = cudaStreamWaitEvent(h->io_in, h->ev_in_free, 0);
  if (e == cudaSuccess) e = swgb::guard_state_write(h, h->stage_in, h->io_in);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->stage_in, host, bytes, cudaMemcpyHostToDevice, h->io_in);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_in_done, h->io_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_in_done, 0);
  if (e != cudaSuccess) return io_cuda(e, "set_spins_async");
  std::swap(h->lat.spins, h->stage_in);
  e = cudaEventRecord(h->ev_in_free, h->stream);
  if (e != cudaSuccess) return io_cuda(e, "set_spins_async");
  h->in_free_set = true;
  return SW_OK;
}

int sw_get_spins_async(sw_handle* h, void* host, size_t bytes) {
  int rc = check_io_args(h, host, bytes);
  if (rc != SW_OK) return rc;
  cudaError_t e = ensure_io(h);
  if (e != cudaSuccess) return io_cuda(e, "asynchronous I/O setup");
  const int b = h->lat.spins == h->io_buf[0] ? 0 : 1;
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_state, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_out, h->ev_state, 0);
  // the buffer itself goes to the host; its next write waits for ev_down
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, h->lat.spins, bytes, cudaMemcpyDeviceToHost, h->io_out);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_down[b], h->io_out);
  if (e != cudaSuccess) return io_cuda(e, "get_spins_async");
  h->down_wait[b] = true;
  return SW_OK;
}

int sw_get_record_async(sw_handle* h, uint64_t sweep, sw_record* host) {
  if (!h || !host) return io_fail(SW_ERR_BAD_ARG, "NULL argument");
  if (sweep == 0 || sweep > h->sweep) return io_fail(SW_ERR_RANGE, "sweep not run yet");
  if (h->sweep - sweep >= (uint64_t)h->meas.series_cap)
    return io_fail(SW_ERR_RANGE, "sweep record no longer retained");
  cudaError_t e = ensure_io(h);
  if (e != cudaSuccess) return io_cuda(e, "asynchronous I/O setup");
  if (h->pending == sweep) e = swgb::flush_pending(h);
  static_assert(sizeof(swgb::Record) == sizeof(sw_record), "record layout");
  const swgb::Record* ring = static_cast<const swgb::Record*>(h->meas.series);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_rec, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->io_out, h->ev_rec, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, ring + (sweep % (uint64_t)h->meas.series_cap), sizeof(sw_record),
                        cudaMemcpyDeviceToHost, h->io_out);
  return e == cudaSuccess ? SW_OK : io_cuda(e, "get_record_async");
}

int sw_wait_io(sw_handle* h) {
  if (!h) return io_fail(SW_ERR_BAD_ARG, "NULL handle");
  cudaError_t e = swgb::wait_io(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? SW_OK : io_cuda(e, "wait_io");
}

}  // extern "C"
