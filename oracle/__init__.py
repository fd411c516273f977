"""FP64 CPU oracle of the KISS-Matcher front end (arXiv 2409.15615).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs use it.  The product path (the CUDA
library and its Python binding) never imports, calls or links anything here,
and nothing here imports the product.

The heavy loops live in ``kmx_oracle.c`` (plain C, FP64, compiled by
``oracle.build``); this module marshals numpy arrays and adds the parts of the
method downstream of matching (ratio filter, pairwise-invariant graph, max
k-core, GNC-TLS pose) that the end-to-end check needs.

Every function cites the passage of the paper it follows; the readings of the
passages the paper leaves open are listed at the top of ``kmx_oracle.c``.
"""
from .core import (  # noqa: F401
    OracleParams,
    load,
    voxelize,
    radius_search,
    eig3_jacobi,
    normals,
    valid_filter,
    pair_features,
    feature_bin,
    spfh,
    fpfh,
    faster_pfh,
    classic_fpfh,
    nearest,
    mutual_match,
    front_end,
)
from .registration import (  # noqa: F401
    ratio_filter,
    invariant_graph,
    core_numbers,
    max_kcore,
    horn,
    gnc_tls,
    register,
    pose_errors,
    is_success,
)
