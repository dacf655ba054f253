// Launchers of the anisotropic lookup shared by aniso.cu and lookup.cu.
// They validate nothing: the C-ABI entry point has checked every argument.
#pragma once

#include "htex_internal.h"

// Anisotropic lookups (aniso.cu).
htex_status htex_launch_aniso(const htex_textures* t, const htex_query_aniso* q, int64_t n, int32_t kmax,
                              float* out, htex_stream stream, int32_t* d_status);

// The same on queries sorted by halfedge range (HTEX_LOOKUP_BIN, lookup.cu),
// chunk by chunk, results gathered back into query order; unsorted for
// pools that fit L2.
htex_status htex_launch_aniso_sorted(const htex_textures* t, const htex_query_aniso* q, int64_t n, int32_t kmax,
                                     float* out, htex_stream stream, int32_t* d_status);
