// Host-side scene construction (see scene_build.cpp).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/wost.h"
#include "wost_internal.h"

namespace wost {

struct HostTree {
    std::vector<float4> nodes, cones, prims, data;
    std::vector<float4> data_minus;  // - side corner data (double-sided records; empty if none)
    std::vector<uint8_t> sided;      // per record: 1 = double-sided (empty if none is)
    std::vector<int32_t> ids;
    uint32_t root = WOST_EMPTY_REF;
    float root_lo[3] = {0, 0, 0}, root_hi[3] = {0, 0, 0};
    float4 root_cone = {0, 0, 1, -1};
    int n_prims = 0, n_nodes = 0, depth = 0;
    // 8-wide layout of the same tree (same primitive records and order)
    std::vector<float4> wnodes, wcones;
    uint32_t wroot = WOST_EMPTY_REF;
    int wn_nodes = 0, wdepth = 0;
    std::vector<std::vector<int>> wslots;  // build-time only: binary children of each wide node
    std::vector<int> wide_of;
};

struct HostScene {
    int dim = 0;
    HostTree D, N, S;
    FieldView g{}, h{}, f{};
    std::vector<float> grid, grid_unused;
    int64_t n_dirichlet = 0, n_neumann = 0, n_silhouette = 0, n_dropped = 0;
    float lo[3], hi[3];
    double build_seconds = 0;
};

// Validates the description and builds every host-side array.  Returns an
// empty string on success, else the reason for rejecting the input.
std::string build_scene(const wost_scene_desc &desc, HostScene &out);

// Structural checks of the built hierarchies (scene_check.cpp): empty string
// when they hold, else the first violation.
std::string check_scene(const HostScene &scene);

}  // namespace wost
