/*
 * Measurement aids of libfte_gb300 (the paper has no counterpart: they are not
 * steps of the method).  They give the ceilings against which the transport
 * kernel's gather throughput is reported: the read bandwidth of the memory level
 * that serves a gather, measured with the gather's own load shapes.
 * Conventions as in fte.h (status codes, fte_last_error, DEVICE pointers owned by
 * the caller, asynchronous on `stream`).
 */
#ifndef FTE_PROBE_H
#define FTE_PROBE_H

#include "fte.h"

#ifdef __cplusplus
extern "C" {
#endif

/* `threads` threads (a multiple of 256) each read `loads` pseudo-random 32-byte
   sectors of `buf` (DEVICE, 32-byte aligned, `bytes` >= 32) bypassing L1, and write
   one float each to dev_out (DEVICE, `threads` floats).  Timing it gives the
   random-sector read bandwidth of the level holding `buf` (L2 when `bytes` fits in
   L2). */
fte_status fte_probe_sectors(const void* buf, size_t bytes, int threads, int loads, float* dev_out,
                             void* stream);

/* The transport kernel's record loads from a buffer small enough to stay in L1:
   `buf` (DEVICE, 32-byte aligned) holds `bytes` / 96 FP32 cell records of FTE_REC
   floats; each of `threads` threads (a multiple of 256) reads the 18 stored fields
   of `records` consecutive records with the transport kernel's load instructions
   (two 32-byte and one 8-byte non-coherent loads per record, 72 bytes), lane l of
   a warp starting at record (w * 7 + l % spread) of the warp's walk (spread 1: all
   lanes of a warp read the same records, as lanes sharing an interpolation stencil
   after reordering do); dev_out (DEVICE, `threads` floats) receives one value per
   thread.  Delivered bytes = threads * records * 72.  EINVAL for fewer than 64
   records in `buf`, spread outside [1, 32] or records < 1. */
fte_status fte_probe_gather_l1(const void* buf, size_t bytes, int threads, int records, int spread,
                               float* dev_out, void* stream);

/* Step-kernel launch timing for roofline accounting.  capacity > 0: from now on,
   every step-kernel launch of fte_advance (up to `capacity` of them) is bracketed by
   two CUDA events recorded on the stream of that launch (not while that stream is
   being captured); the events are created here on the current device.  capacity 0:
   stop and release them.  Process-wide state, guarded by a mutex. */
fte_status fte_probe_step_timing(int capacity);

/* Synchronises the recorded events and writes host_ms[2 i], host_ms[2 i + 1] (HOST,
   room for `capacity` launches): the start and end of recorded launch i in
   milliseconds after the start of the first one; *count = launches recorded.  Then
   forgets them (recording goes on while enabled).  ENOMEM if more than `capacity`
   launches were recorded (*count is set). */
fte_status fte_probe_step_intervals(double* host_ms, int capacity, int* count);

#ifdef __cplusplus
}
#endif
#endif
