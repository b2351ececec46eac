"""msRep SpMV hot path (arXiv 2209.07552) for one GB300 (sm_103a).

pCSR / pCSC / pCOO partitioning (Alg. 2, 4, 6), SpMV over the partitions
with the partial-sum merge of split rows (Alg. 3, 5, 7), in hand-written
CUDA behind the C ABI of include/msrep.h.  ``native`` is the Python binding
of that ABI; ``inputs`` synthesises seeded test and benchmark matrices.
"""
from .native import (MSREP_BF16, MSREP_COMP_ALL, MSREP_COMP_NONE, MSREP_COO,
                     MSREP_COO_BY_COL, MSREP_COO_UNSORTED,
                     MSREP_STREAM_TMA, msrep_device_status, msrep_wait_selftest,
                     MSREP_CSC, MSREP_CSR, MSREP_F32, MSREP_F64, MSREP_VALIDATE,
                     MSREP_PART_MERGE_PATH, MSREP_PART_ROW_BLOCK, MSREP_SCHED_PER_PARTITION,
                     DeviceMatrix, DevicePartition, MsrepError, alloc_workspace,
                     msrep_partition, msrep_partition_coo, msrep_partition_csc,
                     msrep_partition_csr, msrep_partition_local_bound,
                     msrep_plan_size, msrep_spmv, msrep_spmv_workspace_size,
                     msrep_spmm, msrep_spmm_workspace_size, MSREP_SPMM_MAX_K,
                     msrep_tile_supported, msrep_version, DeviceBatch,
                     msrep_autotune, msrep_batch_plan_size, msrep_spmv_batched,
                     msrep_tune_default, Server, ServeTicket,
                     msrep_serve_config_default)

__all__ = [n for n in dir() if n.startswith(("msrep_", "MSREP_"))] + [
    "DeviceMatrix", "DevicePartition", "DeviceBatch", "MsrepError", "alloc_workspace",
    "Server", "ServeTicket"]
