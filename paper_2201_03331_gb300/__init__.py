"""GB300 exhaustive epistasis search (Fiuncho's hot path) behind a C ABI.

The package is a thin Python face over ``libfiuncho.so``; see
``include/fiuncho.h`` for the contract of every entry point.  Build the
library with :func:`paper_2201_03331_gb300.build.build`.
"""
from ._binding import (  # noqa: F401
    FC_EINVAL,
    FC_ENODEV,
    FC_ENOMEM,
    FC_ERANGE,
    FC_ECUDA,
    FC_ETIMEOUT,
    FC_KMAX_SEARCH,
    FC_KMAX_TABLES,
    FC_MAX_LIST,
    FC_OK,
    FiunchoError,
    Handle,
    LIB_PATH,
    fc_free,
    fc_info,
    fc_last_search_kind,
    fc_pairs_dense,
    fc_last_error,
    fc_load,
    fc_load_batch,
    fc_batch_info,
    fc_search_batch,
    fc_search_job,
    fc_load_device,
    fc_num_combinations,
    fc_rank,
    fc_scores,
    fc_search,
    fc_search_static,
    fc_set_stream,
    fc_strerror,
    fc_tables,
    fc_sweep_tables,
    fc_timing,
    fc_unrank,
    library,
)
