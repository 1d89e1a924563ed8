"""One rank of the two-rank replica check in test_replicas.py (launched by
torch.distributed.run with the gloo backend on the host): each rank reports
its environment, the slowest rank's step time and the whole job's rate as
computed by the package's replica helpers."""
import json
import os
import sys

import torch
import torch.distributed as dist

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2306_04467_gb300 import replicas  # noqa: E402

ws, rank, local = replicas.dist_env()
dist.init_process_group("gloo")
ms = 3.0 + 2.0 * rank                      # this rank's step time
slowest = replicas.max_over_ranks(ms, torch.device("cpu"))
rate = replicas.job_rate(1000.0, slowest, ws)
# one file per rank (the ranks share the launcher's stdout)
with open(os.path.join(os.environ["REPLICA_OUT"], "rank%d.json" % rank), "w") as f:
    json.dump({"rank": rank, "ws": ws, "local": local, "ms": ms, "slowest": slowest, "rate": rate}, f)
dist.barrier()
dist.destroy_process_group()
