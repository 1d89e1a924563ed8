"""One rank of the two-rank ensemble-sharding check in test_replicas.py
(torch.distributed.run, gloo backend, on the host): the ranks split a small
seeded ensemble by triangle count, each advances its own instances with the
FP64 oracle (standing in for a rank's GPU), and every rank gathers all the
instances' masses and times."""
import json
import os
import sys

import numpy as np
import torch.distributed as dist

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle.oracle import Oracle  # noqa: E402
from paper_2306_04467_gb300 import inputs, replicas  # noqa: E402

ws, rank, local = replicas.dist_env()
dist.init_process_group("gloo")
ns = [4, 7, 5, 6, 3]
sizes = [2 * n * n for n in ns]
mine = replicas.partition_instances(sizes, ws)[rank]
local_res = {}
for i in mine:
    prob = inputs.ensemble_member(ns[i], seed=100 + i)
    o = Oracle.from_problem(prob)
    o.advance(4)
    local_res[i] = [float(x) for x in o.mass()] + [o.t]
allres = replicas.gather_instance_results(local_res, len(ns))
with open(os.path.join(os.environ["REPLICA_OUT"], "shard%d.json" % rank), "w") as f:
    json.dump({"rank": rank, "mine": mine, "all": allres}, f)
dist.barrier()
dist.destroy_process_group()
