// marker_src.cuh -- the marker source a step's IB kernel may read its
// markers from (fg_step_markers, fg_step_io).
#pragma once

namespace fl {

// The coming step's marker positions and velocities in the caller's own
// arrays (float [total markers][3] each, the environments' markers one after
// the other: the compact numbering), posted by fg_step_markers.  While valid
// is set, the step's IB kernel reads the markers there and copies them into
// the domain's marker arrays on the way (instead of a copy launch before the
// step); the step's reduction clears valid.
struct MarkerSrc {
    const float* X;
    const float* U;
    int valid;
};

}  // namespace fl
