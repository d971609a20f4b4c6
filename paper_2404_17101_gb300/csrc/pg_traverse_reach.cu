// pg_traverse_reach.cu -- the reachability (REACH) instantiation of the
// persistent traversal kernel of pg_traverse.cu, built as a translation unit
// of its own so that the two instantiations compile in parallel.  It defines
// pg_launch_traverse_reach; pg_traverse.cu defines the BFS launches.
#define PG_TRAVERSE_REACH_TU 1
#include "pg_traverse.cu"
