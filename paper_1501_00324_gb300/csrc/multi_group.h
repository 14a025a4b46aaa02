// Lockstep multi-RHS solve groups for the solve server (multi_cg.cu).
//
// A group is the lockstep CG of cg_solve_multi on one matrix with a fixed width
// kw whose columns are filled and emptied while it runs: a request added to a
// free column starts at the group's next outer step (those come on the fixed
// grid of 8 * check_every inner iterations, or at once when no column
// iterates), and a column's x is read out at the outer step that finishes it.
// Because a column's iterates depend only on its own data and the grid, a
// request's x is bitwise the same as cg_solve_multi of that right-hand side
// with the same width, whatever else the group holds.
#pragma once

#include <cstdint>
#include <vector>

#include "internal.h"

namespace fespmv {

struct MultiGroup;

struct GroupDone {
    int64_t tag = 0;
    cg_result res{};
    std::vector<double> x;   // input numbering
};

// The width the server uses for a matrix when asked to choose: 32 columns for
// small matrices, fewer as the n x kw vectors grow (at most 2^21 entries, at
// least 4 columns).
int group_width_auto(const fespmv_mat* A);
// Device bytes a group of width kw needs.
int64_t group_bytes(const fespmv_mat* A, int kw);
// A group for requests with options `o` (precision FESPMV_CG_F64 or
// FESPMV_CG_F32_REFINE, flags FESPMV_CG_RELIABLE / FESPMV_CG_NO_PRECOND, the
// same check_every); BREAKDOWN for a bad diagonal, UNSUPPORTED as cg_solve_multi.
int group_create(fespmv_mat* A, int kw, const cg_options& o, MultiGroup** out);
void group_destroy(MultiGroup* g);
int64_t group_device_bytes(const MultiGroup* g);
bool group_matches(const MultiGroup* g, const cg_options& o);
int group_free_columns(const MultiGroup* g);
int group_width_of(const MultiGroup* g);
// No column in use and no work enqueued.
bool group_empty(const MultiGroup* g);
// Put a request (b in the input numbering, host, copied) in a free column.
int group_add(MultiGroup* g, int64_t tag, const double* b, const cg_options& o);
// Advance without blocking on the GPU: appends the requests finished by this
// step to `done`; *progress tells whether anything happened.
int group_step(MultiGroup* g, bool* progress, std::vector<GroupDone>& done);

}  // namespace fespmv
